// mpr_batch_kernels.cuh -- device code of the batched launch: many independent gap-filling
// problems in one launch (included by the per-storage translation units mpr_batch_<type>.cu, which
// instantiate the kernels of one spin storage type each so the four compile in parallel, and by
// mpr_batch.cu for the list compaction of its finish kernel).
//
// Every problem of a batch runs the whole method of Sec. 2 -- temperature tuning (bisection on
// e_b(T) = e_s), equilibration, sampling -- inside one launch. Each iteration is one hybrid sweep
// of every problem that is not finished: red tiles of all active problems, then black tiles. The
// block that completes the last black tile of a problem (per-problem arrival counter) sums that
// problem's tile energy partials in a fixed order and advances its state machine: probe
// bookkeeping and the bisection step in FP64 (the same arithmetic as the single-problem host
// loop), then equilibration, sampling, done. Problems of uneven size finish at different
// iterations; their tiles leave the list.
//
// Persistent mode: one cooperative kernel whose blocks meet at a grid barrier between passes; the
// barrier spins with a time limit, and a wait that runs out sets an error word, every block
// leaves, the kernel ends normally and the host reports MPR_ERR_DEVICE_TIMEOUT.
#pragma once

#include <type_traits>

#include "mpr.h"
#include "mpr_batch.h"
#include "mpr_tile_f32.cuh"

namespace mpr {
namespace batch {
namespace {

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
    d.nfill = __ldcg(&P.d.nfill);
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
        d.nfill += 1;
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
// arguments are a pointer and scalars, so nothing passes through local memory. ks (SCHED): the
// kernel parameter holding the batch's Philox round keys (one seed for every problem), so they
// enter the rounds as constant operands; the counter-dependent half of round 1 is formed per tile.
template <typename S, int R, int TJ, bool MEASURE, int SAMPLE, bool SCHED, int QM = 0>
__device__ __forceinline__ void tile_body(const Args* __restrict__ A, int t, int p, int colour,
                                          int tx, int ty, const PhiloxSched* ks)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const Prob& P = A->prob[p];
    SweepArgs a{};
    a.own = static_cast<char*>(A->ang) + (size_t)P.ang_off[colour] * sizeof(S);
    a.other = static_cast<const char*>(A->ang) + (size_t)P.ang_off[colour ^ 1] * sizeof(S);
    a.mbits = A->mb + P.mb_off[colour];
    a.acc = A->acc ? A->acc + P.acc_off[colour] : nullptr;
    a.acc_hi = A->acc_hi ? A->acc_hi + P.acc_off[colour] : nullptr;
    a.acc_lo = A->acc_lo ? A->acc_lo + P.acc_off[colour] : nullptr;
    a.part32 = A->part32 ? A->part32 + P.acc_off[colour] : nullptr;
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
    a.nl2eTf = -1.4426950408889634f * a.invTf;
    if constexpr (SCHED) {
        a.ph = *ks;
        const uint64_t m = (uint64_t)0xCD9E8D57u * a.sweep;
        a.ph.a = (uint32_t)(m >> 32) ^ a.seed_lo;
        a.ph.b = (uint32_t)m;
        a.ph.c = (((uint32_t)p << 8) | (kTagMetropolis << 1) | (uint32_t)colour) ^ a.seed_hi;
    }
    void* eslot = MEASURE ? static_cast<char*>(A->epart) + (size_t)t * (A->energy_f32 ? 4 : 8) : nullptr;
    // PDL: own values first, then the wait for the previous kernel (a no-op unless it hangs on a
    // programmatic edge, and in the persistent kernel), then the release of the next one
    sweep_tile<S, R, MEASURE, SAMPLE, SCHED, true, false, TJ, QM>(
        a, tx, ty, *reinterpret_cast<TileSmem<R, TJ>*>(dsm), eslot);
}

// Folds the int32 sample partials of this thread's sites of tile (tx, ty) into the FP64 sums
// (the sites whose partials the thread itself added to in sweep_tile: its R rows, its 4 columns):
// acc += v * 2^-24 is exact, so the sums are the bits that adding every sampled angle in FP64
// gives (the single handle folds the same way, in a separate kernel).
template <int R, int TJ>
__device__ __forceinline__ void fold_tile(const Args* __restrict__ A, const Prob& P, int colour,
                                          int tx, int ty)
{
    constexpr int TY = tile_rows<R, TJ>();
    const int lc = threadIdx.x % Lanes<TJ>::kPerRow, lr = threadIdx.x / Lanes<TJ>::kPerRow;
    const int row0 = (threadIdx.y * Lanes<TJ>::kRows + lr) * R;
    const int jb = tx * TJ + 4 * lc;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int y = ty * TY + row0 + i;
        if (y >= P.Ly) break;
        const long long idx = P.acc_off[colour] + (long long)y * P.pitch + jb;
        int4* pp = reinterpret_cast<int4*>(A->part32 + idx);
        const int4 v = *pp;
        if ((v.x | v.y | v.z | v.w) == 0) continue;
        double2* q = reinterpret_cast<double2*>(A->acc + idx);
        double2 s0 = q[0], s1 = q[1];
        s0.x += (double)v.x * 0x1.0p-24;
        s0.y += (double)v.y * 0x1.0p-24;
        s1.x += (double)v.z * 0x1.0p-24;
        s1.y += (double)v.w * 0x1.0p-24;
        q[0] = s0;
        q[1] = s1;
        *pp = make_int4(0, 0, 0, 0);
    }
}

template <typename S, int R, int TJ, bool MEASURE, int SAMPLE>
__device__ __noinline__ void tile_fn(const Args* __restrict__ A, int t, int p, int colour, int tx,
                                     int ty)
{
    tile_body<S, R, TJ, MEASURE, SAMPLE, false>(A, t, p, colour, tx, ty, nullptr);
    if constexpr (SAMPLE == 3) {
        // sample `step` of this run (the bookkeeping advances it after both passes): 16 int32
        // partials of angles below 8 stay below 2^31, so fold after every 16th and the last
        const Prob& P = A->prob[p];
        const int step = __ldcg(&P.d.step);
        if ((step & 15) == 15 || step == A->samples - 1) fold_tile<R, TJ>(A, P, colour, tx, ty);
    }
}

// FP16 storage: every stored angle is a multiple of 2^-24, so sampling adds exact int32 partials
// (A->part32) instead of FP64 values.
template <typename S> constexpr bool kFix = std::is_same<S, __half>::value;

// The variant of a tile of shape (R, TJ) for this pass: plain inlined (QM as in sweep_tile), the
// others as calls.
template <typename S, int R, int TJ, int QM>
__device__ __forceinline__ void tile_variant(const Args* __restrict__ A, int t, int p, int colour,
                                             int tx, int ty, bool measure, bool sample,
                                             const PhiloxSched& ks)
{
    if (!measure && !sample) {
        tile_body<S, R, TJ, false, 0, true, QM>(A, t, p, colour, tx, ty, &ks);
    } else if (measure && !sample) {
        tile_fn<S, R, TJ, true, 0>(A, t, p, colour, tx, ty);
    } else if (!measure) {
        if (kFix<S> && A->part32) tile_fn<S, R, TJ, false, (kFix<S> ? 3 : 1)>(A, t, p, colour, tx, ty);
        else if (A->acc_kind == 0) tile_fn<S, R, TJ, false, 1>(A, t, p, colour, tx, ty);
        else tile_fn<S, R, TJ, false, 2>(A, t, p, colour, tx, ty);
    } else {
        if (kFix<S> && A->part32) tile_fn<S, R, TJ, true, (kFix<S> ? 3 : 1)>(A, t, p, colour, tx, ty);
        else if (A->acc_kind == 0) tile_fn<S, R, TJ, true, 1>(A, t, p, colour, tx, ty);
        else tile_fn<S, R, TJ, true, 2>(A, t, p, colour, tx, ty);
    }
}

// Tile t of problem p. The plain pass (no energy, no sampling: most passes) is inlined; the rarer
// variants are calls.
template <typename S, int R, int TJ, int QM = 0>
__device__ __forceinline__ void do_tile(const Args* __restrict__ A, int t, int p, int colour,
                                        TileSmem<R, TJ>& sm, const PhiloxSched& ks)
{
    Prob& P = A->prob[p];
    const int ph = __ldcg(&P.d.phase);
    if (ph == kDone) return;
    const bool measure = colour == 1 && (ph == kProbeMeasure || ph == kRunSample);
    const bool sample = ph == kRunSample;
    const int i = t - P.tile_base;
    const int tx = i % P.ntx, ty = i / P.ntx;
    // 128-column tiles with an even row count per thread: a problem whose last tile column holds
    // at most 64 columns runs that column with the 64-column code of the same height (tile column
    // 2 tx in 64-column units), wasting half as much of the tile; with a row count per thread
    // divisible by 4, one of at most 32 columns runs with the 32-column code (tile column 4 tx)
    constexpr bool kTail = TJ == 128 && R % 2 == 0;
    constexpr bool kTail32 = TJ == 128 && R % 4 == 0;
    const bool last = tx == P.ntx - 1;
    if constexpr (kTail32) {
        if (last && P.tail == 32) {
            tile_variant<S, R / 4, 32, QM>(A, t, p, colour, 4 * tx, ty, measure, sample, ks);
        } else if (last && P.tail == 64) {
            tile_variant<S, R / 2, 64, QM>(A, t, p, colour, 2 * tx, ty, measure, sample, ks);
        } else {
            tile_variant<S, R, TJ, QM>(A, t, p, colour, tx, ty, measure, sample, ks);
        }
    } else if constexpr (kTail) {
        if (last && P.tail == 64)
            tile_variant<S, R / 2, 64, QM>(A, t, p, colour, 2 * tx, ty, measure, sample, ks);
        else
            tile_variant<S, R, TJ, QM>(A, t, p, colour, tx, ty, measure, sample, ks);
    } else {
        tile_variant<S, R, TJ, QM>(A, t, p, colour, tx, ty, measure, sample, ks);
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
template <typename S, int R, int TJ>
__device__ __forceinline__ void colour_pass(const Args* __restrict__ A, const int2* list, int n,
                                            int colour, TileSmem<R, TJ>& sm, volatile int* s_k,
                                            const PhiloxSched& ks)
{
    if (threadIdx.x == 0 && threadIdx.y == 0) *s_k = (int)atomicAdd(&A->ctl->work[colour], 1u);
    __syncthreads();
    int k = *s_k;
    while (k < n) {
        __syncthreads();   // every thread has read s_k
        if (threadIdx.x == 0 && threadIdx.y == 0) *s_k = (int)atomicAdd(&A->ctl->work[colour], 1u);
        const int2 e = __ldcg(list + k);
        do_tile<S, R, TJ>(A, e.x, e.y, colour, sm, ks);
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

template <typename S, int R, int TJ>
__global__ void __launch_bounds__(256, 3) batch_kernel(const Args* __restrict__ A,
                                                        const PhiloxSched ks)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    TileSmem<R, TJ>& sm = *reinterpret_cast<TileSmem<R, TJ>*>(dsm);
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
        colour_pass<S, R, TJ>(A, list, n, 0, sm, &s_k, ks);
        if (!grid_barrier(ctl, expected, &s_err, &ctl->work[0])) return;
        colour_pass<S, R, TJ>(A, list, n, 1, sm, &s_k, ks);
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

// ---- graph mode: one launch of a CUDA graph whose while-loop node repeats a red and a black
// pass kernel and the finish kernel (mpr_batch.cu) on the device until every problem is done.
// Each pass kernel runs one tile per block (the hardware scheduler overlaps many blocks, hiding
// each tile's load latency); the finish kernel shrinks the tile list and sets the loop
// condition. No grid barrier, no spin wait.

// Compiled for 4 resident blocks per SM: the inlined plain tile (most passes) fits 64 registers;
// the rarer energy and sampling variants are calls that may spill.
// QM: 2 for the batch's q = 1/2 (16-bit storages), else 0 (see sweep_tile).
// The tile list, its length and the problems' phases were last written by the finish kernel and
// the black pass of the previous sweep, which have completed before a red pass starts (the red
// pass is the first node of the loop body) and before a black pass starts (it hangs on the red
// pass, which released it only after its own wait): a block reads them before its wait.
template <typename S, int R, int TJ, int QM>
__global__ void __launch_bounds__(256, 4) pass_kernel(const Args* __restrict__ A, int colour,
                                                       const PhiloxSched ks)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const Ctl* ctl = A->ctl;
    const int k = blockIdx.x;
    if (k >= __ldcg(&ctl->n_list)) return;
    const int2 e = __ldcg(A->lists + (size_t)__ldcg(&ctl->list_sel) * A->ntiles + k);
    do_tile<S, R, TJ, QM>(A, e.x, e.y, colour, *reinterpret_cast<TileSmem<R, TJ>*>(dsm), ks);
}


// The kernels of storage type S for tile shape s (kShape).
template <typename S, int R, int TJ>
Kernels entry()
{
    const void* qh = nullptr;
    if constexpr (sizeof(S) == 2) qh = reinterpret_cast<const void*>(&pass_kernel<S, R, TJ, 2>);
    return Kernels{reinterpret_cast<const void*>(&pass_kernel<S, R, TJ, 0>),
                   reinterpret_cast<const void*>(&batch_kernel<S, R, TJ>), sizeof(TileSmem<R, TJ>),
                   qh};
}

template <typename S>
Kernels table(int s)
{
    switch (s) {
    case 0: return entry<S, 1, 128>();
    case 1: return entry<S, 2, 128>();
    case 2: return entry<S, 4, 128>();
    case 3: return entry<S, 1, 64>();
    case 4: return entry<S, 2, 64>();
    default: return Kernels{nullptr, nullptr, 0, nullptr};
    }
}

}  // namespace
}  // namespace batch
}  // namespace mpr
