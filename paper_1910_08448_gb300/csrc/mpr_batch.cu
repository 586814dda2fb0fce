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
__device__ bool grid_barrier(Ctl* ctl, unsigned expected, volatile int* s_err, unsigned* reset)
{
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        volatile unsigned* gen = &ctl->bar_gen;
        volatile int* err = &ctl->err;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
        if (arrived == expected - 1) {
            // last arrival: every block is done with the pass, its work counter can restart
            atomicExch(reset, 0u);
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
    if (d.phase == kDone) {
        atomicSub(&A.ctl->n_active, 1);
        atomicExch(&A.ctl->changed, 1);
    }
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

// The sweep's bond sum of problem P from its tile partials, by the whole block: thread t adds
// tiles t, t + 256, ... and a shared-memory tree combines the 256 sums -- the same fixed order as
// the single-problem reduction, so both paths give the same bits. Result valid in thread 0.
template <typename E>
__device__ double block_energy(const Prob& P, const Args& A, E* red)
{
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const E* ep = static_cast<const E*>(A.epart) + P.tile_base;
    E s = (E)0;
    for (int i = tid; i < P.ntiles; i += 256) s += __ldcg(ep + i);
    red[tid] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    return (double)red[0];
}

// After the last black tile of problem P in this sweep (one thread): the state machine, given the
// sweep's raw bond sum when the sweep was measured.
__device__ void bookkeeping(Prob& P, const Args& A, double raw)
{
    Dyn d;
    load_dyn(P, d);
    const int ph = d.phase;
    double e = 0.0;
    if (ph == kProbeMeasure || ph == kRunSample) e = -raw / P.Nb;
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
            if (d.phase == kDone) {
                atomicSub(&A.ctl->n_active, 1);
                atomicExch(&A.ctl->changed, 1);
            }
        }
        break;
    case kRunSample:
        d.esamp += e;
        d.nsamples += 1;
        if (++d.step >= A.samples) {
            d.phase = kDone;
            atomicSub(&A.ctl->n_active, 1);
            atomicExch(&A.ctl->changed, 1);
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

// Builds the sweep arguments of tile t (colour `colour`) and runs it. One function per variant,
// not inlined, so every variant gets its own register allocation within the kernel's budget; the
// arguments are a pointer and scalars, so nothing passes through local memory.
template <typename S, int R, bool MEASURE, int SAMPLE>
__device__ __forceinline__ void tile_body(const Args* __restrict__ A, int t, int p, int colour)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const Prob& P = A->prob[p];
    SweepArgs a;
    a.own = static_cast<char*>(A->ang) + (size_t)P.ang_off[colour] * sizeof(S);
    a.other = static_cast<const char*>(A->ang) + (size_t)P.ang_off[colour ^ 1] * sizeof(S);
    a.mbits = A->mb + P.mb_off[colour];
    a.acc = A->acc ? A->acc + P.acc_off[colour] : nullptr;
    a.acc_hi = A->acc_hi ? A->acc_hi + P.acc_off[colour] : nullptr;
    a.acc_lo = A->acc_lo ? A->acc_lo + P.acc_off[colour] : nullptr;
    a.epart = A->epart;
    a.Lx = P.Lx;
    a.Ly = P.Ly;
    a.Lxh = P.Lxh;
    a.pitch = P.pitch;
    a.mpitch = P.mpitch;
    a.colour = colour;
    a.flags = A->energy_f32 ? kEnergyF32 : 0;
    a.seed_lo = A->seed_lo;
    a.seed_hi = A->seed_hi;
    // state written by other blocks' bookkeeping: read at L2, not through this SM's L1
    a.sweep = __ldcg(&P.d.sweep);
    a.problem = (uint32_t)p;
    a.q = A->q;
    a.T = 0.0;
    a.invT = 0.0;        // the FP32 tile uses qf and invTf only
    a.qf = A->qf;
    a.invTf = __ldcg(&P.d.invTf);
    const int i = t - P.tile_base;
    void* eslot = MEASURE ? static_cast<char*>(A->epart) + (size_t)t * (A->energy_f32 ? 4 : 8) : nullptr;
    sweep_tile<S, R, MEASURE, SAMPLE, false>(a, i % P.ntx, i / P.ntx, *reinterpret_cast<TileSmem<R>*>(dsm),
                                      eslot);
}

template <typename S, int R, bool MEASURE, int SAMPLE>
__device__ __noinline__ void tile_fn(const Args* __restrict__ A, int t, int p, int colour)
{
    tile_body<S, R, MEASURE, SAMPLE>(A, t, p, colour);
}

// Tile t of problem p. The plain pass (no energy, no sampling: most passes) is inlined; the rarer
// variants are calls.
template <typename S, int R>
__device__ __forceinline__ void do_tile(const Args* __restrict__ A, int t, int p, int colour,
                                        TileSmem<R>& sm)
{
    Prob& P = A->prob[p];
    const int ph = __ldcg(&P.d.phase);
    if (ph == kDone) return;
    const bool measure = colour == 1 && (ph == kProbeMeasure || ph == kRunSample);
    const bool sample = ph == kRunSample;
    if (!measure && !sample) {
        tile_body<S, R, false, 0>(A, t, p, colour);
    } else if (measure && !sample) {
        tile_fn<S, R, true, 0>(A, t, p, colour);
    } else if (!measure) {
        if (A->acc_kind == 0) tile_fn<S, R, false, 1>(A, t, p, colour);
        else tile_fn<S, R, false, 2>(A, t, p, colour);
    } else {
        if (A->acc_kind == 0) tile_fn<S, R, true, 1>(A, t, p, colour);
        else tile_fn<S, R, true, 2>(A, t, p, colour);
    }
    if (colour == 1) {
        __shared__ int s_last;
        __syncthreads();   // the tile's partial and spins are written before the arrival counts
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            __threadfence();
            s_last = atomicAdd(&P.tiles_done, 1u) == (unsigned)P.ntiles - 1u;
            if (s_last) __threadfence();
        }
        __syncthreads();
        if (s_last) {   // this block finished the problem's sweep: energy, then state machine
            double raw = 0.0;
            if (measure) {
                raw = A->energy_f32 ? block_energy<float>(P, *A, reinterpret_cast<float*>(&sm.cs[0][0]))
                                    : block_energy<double>(P, *A, reinterpret_cast<double*>(&sm.cs[0][0]));
            }
            if (threadIdx.x == 0 && threadIdx.y == 0) {
                bookkeeping(P, *A, raw);
                __threadfence();
            }
        }
    }
}

// One colour pass over the active tile list: blocks take tiles from a shared counter (largest
// tiles first, so uneven tiles and problems balance); the next index is fetched while the current
// tile runs.
template <typename S, int R>
__device__ __forceinline__ void colour_pass(const Args* __restrict__ A, const int2* list, int n,
                                            int colour, TileSmem<R>& sm, volatile int* s_k)
{
    if (threadIdx.x == 0 && threadIdx.y == 0) *s_k = (int)atomicAdd(&A->ctl->work[colour], 1u);
    __syncthreads();
    int k = *s_k;
    while (k < n) {
        __syncthreads();   // every thread has read s_k
        if (threadIdx.x == 0 && threadIdx.y == 0) *s_k = (int)atomicAdd(&A->ctl->work[colour], 1u);
        const int2 e = __ldcg(list + k);
        do_tile<S, R>(A, e.x, e.y, colour, sm);
        __syncthreads();
        k = *s_k;
    }
}

// Stable compaction of the active tile list (one block): drop the tiles of finished problems.
__device__ void compact_list(const Args* __restrict__ A, const int2* src, int n, int2* dst, int* n_out,
                             int* scan)
{
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int per = (n + 255) / 256;
    const int b = tid * per, e = min(n, b + per);
    int cnt = 0;
    for (int k = b; k < e; ++k) cnt += __ldcg(&A->prob[__ldcg(src + k).y].d.phase) != kDone;
    scan[tid] = cnt;
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int i = 0; i < 256; ++i) {
            const int c = scan[i];
            scan[i] = run;
            run += c;
        }
        *n_out = run;
    }
    __syncthreads();
    int o = scan[tid];
    for (int k = b; k < e; ++k) {
        const int2 t = __ldcg(src + k);
        if (__ldcg(&A->prob[t.y].d.phase) != kDone) dst[o++] = t;
    }
    __threadfence();
    __syncthreads();
}

template <typename S, int R>
__global__ void __launch_bounds__(256, 3) batch_kernel(const Args* __restrict__ A)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    TileSmem<R>& sm = *reinterpret_cast<TileSmem<R>*>(dsm);
    __shared__ int s_err, s_k, s_active, s_changed, s_sel, s_n;
    __shared__ int s_scan[256];
    Ctl* ctl = A->ctl;
    const unsigned expected = gridDim.x + (unsigned)ctl->bar_extra;
    const bool t0 = threadIdx.x == 0 && threadIdx.y == 0;
    if (t0) {
        s_sel = __ldcg(&ctl->list_sel);
        s_n = __ldcg(&ctl->n_list);
    }
    __syncthreads();
    for (int it = 0; it < A->max_iters; ++it) {
        const int2* list = A->lists + (size_t)s_sel * A->ntiles;
        const int n = s_n;
        colour_pass<S, R>(A, list, n, 0, sm, &s_k);
        if (!grid_barrier(ctl, expected, &s_err, &ctl->work[0])) return;
        colour_pass<S, R>(A, list, n, 1, sm, &s_k);
        if (!grid_barrier(ctl, expected, &s_err, &ctl->work[1])) return;
        if (t0) {
            s_active = __ldcg(&ctl->n_active);
            s_changed = __ldcg(&ctl->changed);
            if (blockIdx.x == 0) ctl->iters = it + 1;
        }
        __syncthreads();
        if (s_active <= 0) return;
        if (s_changed) {   // a problem finished in this sweep: shrink the tile list
            if (blockIdx.x == 0) {
                const int sel = s_sel;
                compact_list(A, list, n, A->lists + (size_t)(sel ^ 1) * A->ntiles, &ctl->n_list, s_scan);
                if (t0) {
                    atomicExch(&ctl->list_sel, sel ^ 1);
                    atomicExch(&ctl->changed, 0);
                    __threadfence();
                }
            }
            if (!grid_barrier(ctl, expected, &s_err, &ctl->work[0])) return;
            if (t0) {
                s_sel = __ldcg(&ctl->list_sel);
                s_n = __ldcg(&ctl->n_list);
            }
            __syncthreads();
        }
    }
}

// ---- graph mode: one launch of a CUDA graph whose while-loop node repeats the three kernels
// below on the device until every problem is done. Each pass kernel runs one tile per block (the
// hardware scheduler overlaps many blocks, hiding each tile's load latency); the finish kernel
// shrinks the tile list and sets the loop condition. No grid barrier, no spin wait.

template <typename S, int R>
__global__ void __launch_bounds__(256, 4) pass_kernel(const Args* __restrict__ A, int colour)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const Ctl* ctl = A->ctl;
    const int k = blockIdx.x;
    if (k >= __ldcg(&ctl->n_list)) return;
    const int2 e = __ldcg(A->lists + (size_t)__ldcg(&ctl->list_sel) * A->ntiles + k);
    do_tile<S, R>(A, e.x, e.y, colour, *reinterpret_cast<TileSmem<R>*>(dsm));
}

__global__ void __launch_bounds__(256) finish_kernel(const Args* __restrict__ A,
                                                     cudaGraphConditionalHandle loop)
{
    __shared__ int s_scan[256];
    Ctl* ctl = A->ctl;
    const bool t0 = threadIdx.x == 0 && threadIdx.y == 0;
    if (__ldcg(&ctl->changed)) {   // a problem finished in this sweep: shrink the tile list
        const int sel = __ldcg(&ctl->list_sel);
        compact_list(A, A->lists + (size_t)sel * A->ntiles, __ldcg(&ctl->n_list),
                     A->lists + (size_t)(sel ^ 1) * A->ntiles, &ctl->n_list, s_scan);
        if (t0) {
            ctl->list_sel = sel ^ 1;
            ctl->changed = 0;
        }
    }
    if (t0) {
        const int it = ctl->iters + 1;
        ctl->iters = it;
        __threadfence();
        cudaGraphSetConditional(loop, (__ldcg(&ctl->n_active) > 0 && it < A->max_iters) ? 1u : 0u);
    }
}

template <typename S, int R>
const void* pass_ptr()
{
    return reinterpret_cast<const void*>(&pass_kernel<S, R>);
}

const void* pick_pass(int store, int rows)
{
#define MPR_PICK(S)                                                                           \
    switch (rows) {                                                                           \
    case 1: return pass_ptr<S, 1>();                                                          \
    case 2: return pass_ptr<S, 2>();                                                          \
    case 4: return pass_ptr<S, 4>();                                                          \
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

size_t batch_smem_bytes(int rows)
{
    switch (rows) {
    case 1: return sizeof(f32::TileSmem<1>);
    case 2: return sizeof(f32::TileSmem<2>);
    default: return sizeof(f32::TileSmem<4>);
    }
}

cudaError_t batch_occupancy(int store, int rows, int* blocks_per_sm)
{
    const void* k = batch::pick(store, rows);
    if (!k) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, 256, batch_smem_bytes(rows));
}

cudaError_t batch_launch(int store, int rows, int grid, const batch::Args* args_dev, cudaStream_t st,
                         bool use_graph)
{
    const void* k = batch::pick(store, rows);
    if (!k) return cudaErrorInvalidValue;
    void* params[] = {const_cast<batch::Args**>(&args_dev)};
    if (!use_graph)
        return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(32, f32::kWarps), params,
                                           batch_smem_bytes(rows), st);
    // the same launch as a one-node CUDA graph with a cooperative kernel node
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(k);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(32, f32::kWarps);
    kp.sharedMemBytes = (unsigned)batch_smem_bytes(rows);
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

cudaError_t batch_graph_build(int store, int rows, int max_tiles, const batch::Args* args_dev,
                              cudaGraphExec_t* out)
{
    const void* pass = batch::pick_pass(store, rows);
    if (!pass || max_tiles < 1) return cudaErrorInvalidValue;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle loop;
    e = cudaGraphConditionalHandleCreate(&loop, g, 1u, cudaGraphCondAssignDefault);
    cudaGraphNode_t wnode;
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) {
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = loop;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &cp);
        if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    const int red = 0, black = 1;
    cudaGraphNode_t n_red, n_black, n_fin;
    if (e == cudaSuccess) {
        void* params[] = {const_cast<batch::Args**>(&args_dev), const_cast<int*>(&red)};
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void*>(pass);
        kp.gridDim = dim3(max_tiles);
        kp.blockDim = dim3(32, f32::kWarps);
        kp.sharedMemBytes = (unsigned)batch_smem_bytes(rows);
        kp.kernelParams = params;
        e = cudaGraphAddKernelNode(&n_red, body, nullptr, 0, &kp);
        if (e == cudaSuccess) {
            void* params_b[] = {const_cast<batch::Args**>(&args_dev), const_cast<int*>(&black)};
            kp.kernelParams = params_b;
            e = cudaGraphAddKernelNode(&n_black, body, &n_red, 1, &kp);
        }
    }
    if (e == cudaSuccess) {
        void* params[] = {const_cast<batch::Args**>(&args_dev), &loop};
        cudaKernelNodeParams kp{};
        kp.func = reinterpret_cast<void*>(&batch::finish_kernel);
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32, f32::kWarps);
        kp.sharedMemBytes = 0;
        kp.kernelParams = params;
        e = cudaGraphAddKernelNode(&n_fin, body, &n_black, 1, &kp);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

}  // namespace mpr
