// mpr_batch.cu -- many independent gap-filling problems in one persistent launch.
//
// Every problem of a batch runs the whole method of Sec. 2 -- temperature tuning (bisection on
// e_b(T) = e_s), equilibration, sampling -- inside ONE cooperative kernel launch. Each iteration
// of the kernel is one hybrid sweep of every problem that is not finished: all blocks walk the
// red tiles of all active problems, meet at a grid barrier, walk the black tiles, meet again. The
// block that completes the last black tile of a problem (per-problem arrival counter) sums that
// problem's tile energy partials in a fixed order and advances its state machine: probe
// bookkeeping and the bisection step in FP64 (the same arithmetic as the single-problem host
// loop), then equilibration, sampling, done. Problems of uneven size finish at different
// iterations; their tiles are skipped afterwards.
//
// The grid barrier spins with a time limit: a wait that runs out sets an error word, every block
// leaves, the kernel ends normally and the host reports MPR_ERR_DEVICE_TIMEOUT.
#include "mpr.h"
#include "mpr_batch.h"
#include "mpr_tile_f32.cuh"

namespace mpr {
namespace batch {

using namespace f32;

__device__ __forceinline__ long long globaltimer_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded grid barrier (all blocks co-resident: cooperative launch). Thread 0 arrives, waits with
// a time limit and publishes the error word to its block through shared memory, so every thread
// of a block sees the same answer. The fences on both sides order this block's writes before the
// arrival and the other blocks' writes before this block's later reads. Returns false on error.
__device__ bool grid_barrier(Ctl* ctl, unsigned expected, volatile int* s_err)
{
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        volatile unsigned* gen = &ctl->bar_gen;
        volatile int* err = &ctl->err;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
        if (arrived == expected - 1) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            const long long t0 = globaltimer_ns();
            while (*gen == g) {
                if (*err) break;
                if (globaltimer_ns() - t0 > ctl->timeout_ns) {
                    atomicCAS(&ctl->err, 0, (int)MPR_ERR_DEVICE_TIMEOUT);
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        *s_err = *err;
    }
    __syncthreads();
    return *s_err == 0;
}

// ---- the per-problem state machine (one thread, FP64) --------------------------------------

__device__ void enter_run(Dyn& d, const Args& A)
{
    d.step = 0;
    d.phase = A.equil > 0 ? kRunEquil : (A.samples > 0 ? kRunSample : kDone);
    if (d.phase == kDone) atomicSub(&A.ctl->n_active, 1);
}

__device__ void start_probe(Dyn& d, const Args& A, double T)
{
    d.T = T;
    d.esum = 0.0;
    d.step = 0;
    d.phase = A.n_eq > 0 ? kProbeEquil : kProbeMeasure;
}

// The next bisection probe, or the end of the tuning when the probes are used up.
__device__ void next_mid(Dyn& d, const Args& A)
{
    if (d.np >= A.max_probes) {
        d.T = exp(0.5 * (d.lo + d.hi));
        d.status = MPR_ERR_TUNE_NO_CONVERGE;
        enter_run(d, A);
        return;
    }
    d.mid = 0.5 * (d.lo + d.hi);
    d.kind = 2;
    start_probe(d, A, exp(d.mid));
}

// A probe finished with mean bond energy e: one step of the bisection in log T.
__device__ void probe_done(Dyn& d, const Args& A, double e_s, double e)
{
    const double tol = A.rel_tol * fabs(e_s);
    if (d.kind == 0) {                       // T_lo
        d.np = 1;
        if (fabs(e - e_s) <= tol || e_s < e) { d.T = A.T_lo; enter_run(d, A); return; }
        d.kind = 1;
        start_probe(d, A, A.T_hi);
        return;
    }
    if (d.kind == 1) {                       // T_hi
        d.np = 2;
        if (fabs(e - e_s) <= tol) { d.T = A.T_hi; enter_run(d, A); return; }
        if (e_s > e) { d.T = A.T_hi; d.status = MPR_ERR_TUNE_NO_CONVERGE; enter_run(d, A); return; }
        next_mid(d, A);
        return;
    }
    d.np += 1;                               // bisection midpoint
    if (fabs(e - e_s) <= tol) { enter_run(d, A); return; }
    if (e < e_s) d.lo = d.mid; else d.hi = d.mid;
    if (d.hi - d.lo < A.log_ratio) {
        d.T = exp(0.5 * (d.lo + d.hi));
        enter_run(d, A);
        return;
    }
    next_mid(d, A);
}

__device__ void load_dyn(const Prob& P, Dyn& d)
{
    d.phase = __ldcg(&P.d.phase);
    d.step = __ldcg(&P.d.step);
    d.np = __ldcg(&P.d.np);
    d.kind = __ldcg(&P.d.kind);
    d.status = __ldcg(&P.d.status);
    d.nsamples = __ldcg(&P.d.nsamples);
    d.sweep = __ldcg(&P.d.sweep);
    d.invTf = __ldcg(&P.d.invTf);
    d.T = __ldcg(&P.d.T);
    d.lo = __ldcg(&P.d.lo);
    d.hi = __ldcg(&P.d.hi);
    d.mid = __ldcg(&P.d.mid);
    d.esum = __ldcg(&P.d.esum);
    d.esamp = __ldcg(&P.d.esamp);
    d.site_updates = __ldcg(&P.d.site_updates);
}

// After the last black tile of problem P in this sweep (one thread): the sweep's bond energy from
// the tile partials in tile order, then the state machine.
__device__ void bookkeeping(Prob& P, const Args& A)
{
    Dyn d;
    load_dyn(P, d);
    const int ph = d.phase;
    double e = 0.0;
    if (ph == kProbeMeasure || ph == kRunSample) {
        double raw = 0.0;
        if (A.energy_f32) {
            float s = 0.0f;
            const float* ep = static_cast<const float*>(A.epart) + P.tile_base;
            for (int i = 0; i < P.ntiles; ++i) s += __ldcg(ep + i);
            raw = (double)s;
        } else {
            const double* ep = static_cast<const double*>(A.epart) + P.tile_base;
            for (int i = 0; i < P.ntiles; ++i) raw += __ldcg(ep + i);
        }
        e = -raw / P.Nb;
    }
    d.sweep += 1u;
    d.site_updates += (unsigned long long)P.Np;
    switch (ph) {
    case kProbeEquil:
        if (++d.step >= A.n_eq) { d.phase = kProbeMeasure; d.step = 0; }
        break;
    case kProbeMeasure:
        d.esum += e;
        if (++d.step >= A.n_meas) probe_done(d, A, P.e_s, d.esum / (double)A.n_meas);
        break;
    case kRunEquil:
        if (++d.step >= A.equil) {
            d.step = 0;
            d.phase = A.samples > 0 ? kRunSample : kDone;
            if (d.phase == kDone) atomicSub(&A.ctl->n_active, 1);
        }
        break;
    case kRunSample:
        d.esamp += e;
        d.nsamples += 1;
        if (++d.step >= A.samples) {
            d.phase = kDone;
            atomicSub(&A.ctl->n_active, 1);
        }
        break;
    default:
        break;
    }
    d.invTf = (float)(1.0 / d.T);
    P.d = d;
    P.tiles_done = 0u;
}

// ---- tiles ------------------------------------------------------------------------------------

template <typename S, int R>
__device__ __forceinline__ void do_tile(const Args& A, int t, int colour, TileSmem<R>& sm)
{
    const int p = A.tile_prob[t];
    Prob& P = A.prob[p];
    // state written by other blocks' bookkeeping: read at L2, not through this SM's L1
    const int ph = __ldcg(&P.d.phase);
    if (ph == kDone) return;
    const double T = __ldcg(&P.d.T);
    const unsigned sweep = __ldcg(&P.d.sweep);
    const float invTf = __ldcg(&P.d.invTf);
    SweepArgs a;
    a.own = static_cast<char*>(A.ang) + (size_t)P.ang_off[colour] * sizeof(S);
    a.other = static_cast<const char*>(A.ang) + (size_t)P.ang_off[colour ^ 1] * sizeof(S);
    a.mbits = A.mb + P.mb_off[colour];
    a.acc = A.acc ? A.acc + P.acc_off[colour] : nullptr;
    a.acc_hi = A.acc_hi ? A.acc_hi + P.acc_off[colour] : nullptr;
    a.acc_lo = A.acc_lo ? A.acc_lo + P.acc_off[colour] : nullptr;
    a.epart = A.epart;
    a.Lx = P.Lx;
    a.Ly = P.Ly;
    a.Lxh = P.Lxh;
    a.pitch = P.pitch;
    a.mpitch = P.mpitch;
    a.colour = colour;
    a.flags = A.energy_f32 ? kEnergyF32 : 0;
    a.seed_lo = A.seed_lo;
    a.seed_hi = A.seed_hi;
    a.sweep = sweep;
    a.problem = (uint32_t)p;
    a.q = A.q;
    a.T = T;
    a.invT = 0.0;        // FP64 reciprocal not needed by the FP32 tile
    a.qf = A.qf;
    a.invTf = invTf;
    const int i = t - P.tile_base;
    const int tx = i % P.ntx, ty = i / P.ntx;
    const bool measure = colour == 1 && (ph == kProbeMeasure || ph == kRunSample);
    const bool sample = ph == kRunSample;
    void* eslot = static_cast<char*>(A.epart) + (size_t)t * (A.energy_f32 ? 4 : 8);
    if (!measure && !sample) {
        sweep_tile<S, R, false, 0>(a, tx, ty, sm, nullptr);
    } else if (measure && !sample) {
        sweep_tile<S, R, true, 0>(a, tx, ty, sm, eslot);
    } else if (!measure) {
        if (A.acc_kind == 0) sweep_tile<S, R, false, 1>(a, tx, ty, sm, nullptr);
        else sweep_tile<S, R, false, 2>(a, tx, ty, sm, nullptr);
    } else {
        if (A.acc_kind == 0) sweep_tile<S, R, true, 1>(a, tx, ty, sm, eslot);
        else sweep_tile<S, R, true, 2>(a, tx, ty, sm, eslot);
    }
    if (colour == 1) {
        __syncthreads();   // the tile's partial and spins are written before the arrival counts
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            __threadfence();
            if (atomicAdd(&P.tiles_done, 1u) == (unsigned)P.ntiles - 1u) {
                __threadfence();
                bookkeeping(P, A);
                __threadfence();
            }
        }
    }
}

template <typename S, int R>
__global__ void __launch_bounds__(256, 3) batch_kernel(const Args A)
{
    __shared__ __align__(16) TileSmem<R> sm;
    __shared__ int s_err;
    __shared__ int s_active;
    const unsigned expected = gridDim.x + (unsigned)A.ctl->bar_extra;
    for (int it = 0; it < A.max_iters; ++it) {
        for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) do_tile<S, R>(A, t, 0, sm);
        if (!grid_barrier(A.ctl, expected, &s_err)) return;
        for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) do_tile<S, R>(A, t, 1, sm);
        if (!grid_barrier(A.ctl, expected, &s_err)) return;
        if (threadIdx.x == 0 && threadIdx.y == 0) s_active = __ldcg(&A.ctl->n_active);
        __syncthreads();
        if (s_active <= 0) return;
    }
}

template <typename S, int R>
const void* kernel_ptr()
{
    return reinterpret_cast<const void*>(&batch_kernel<S, R>);
}

const void* pick(int store, int rows)
{
#define MPR_PICK(S)                                                                           \
    switch (rows) {                                                                           \
    case 1: return kernel_ptr<S, 1>();                                                        \
    case 2: return kernel_ptr<S, 2>();                                                        \
    case 4: return kernel_ptr<S, 4>();                                                        \
    default: return nullptr;                                                                  \
    }
    switch (store) {
    case kF64: MPR_PICK(double)
    case kF32: MPR_PICK(float)
    case kF16: MPR_PICK(__half)
    case kBF16: MPR_PICK(__nv_bfloat16)
    default: return nullptr;
    }
#undef MPR_PICK
}

}  // namespace batch

int batch_tile_rows(int rows) { return f32::kWarps * rows; }
int batch_tile_cols() { return f32::kTJ; }

cudaError_t batch_occupancy(int store, int rows, int* blocks_per_sm)
{
    const void* k = batch::pick(store, rows);
    if (!k) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, 256, 0);
}

cudaError_t batch_launch(int store, int rows, int grid, const batch::Args& args, cudaStream_t st,
                         bool use_graph)
{
    const void* k = batch::pick(store, rows);
    if (!k) return cudaErrorInvalidValue;
    void* params[] = {const_cast<batch::Args*>(&args)};
    if (!use_graph)
        return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(32, f32::kWarps), params, 0, st);
    // the same launch as a one-node CUDA graph with a cooperative kernel node
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(k);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(32, f32::kWarps);
    kp.sharedMemBytes = 0;
    kp.kernelParams = params;
    cudaError_t e = cudaGraphCreate(&g, 0);
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&node, g, nullptr, 0, &kp);
    if (e == cudaSuccess) {
        cudaLaunchAttributeValue v{};
        v.cooperative = 1;
        e = cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributeCooperative, &v);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, st);
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    return e;
}

}  // namespace mpr
