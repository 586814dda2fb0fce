// mpr_sweep_f32.cuh -- single-problem colour half-sweep for the FP32 function setting, sweep
// kernel kind 0: one launch per colour pass, one 128 x 32 tile of mpr_tile_f32.cuh per block, 4
// blocks per SM (plain passes), staging with ordinary loads. The hardware block scheduler overlaps
// one block's loads with other blocks' work, and blocks that start and end at different times keep
// the SM's pipes evenly loaded. The alternative kernel kind 1 (TMA-fed, persistent) is in
// mpr_sweep_tma.cu; both apply the same per-site arithmetic, so their results are equal bit for
// bit, and the handle picks the faster one by timing both (mpr_set_sweep_kernel).
//
// Templated on PROP (bounded Metropolis proposals): mpr_sweep_f32.cu instantiates the uniform
// proposal variants, mpr_sweep_f32_prop.cu the bounded ones, so the two compile in parallel.
#pragma once
#include "mpr_tile_f32.cuh"

namespace mpr {
namespace sweep_f32_detail {

using namespace f32;

constexpr int kRows = 4;      // rows per thread of the tiles (128 x 32)

// Compiled for 4 resident blocks per SM (64 registers: no spills with 16-bit spins, a few bytes
// with FP32 spins in the energy and sampling variants); 2 for FP64 spins, whose values take
// twice the registers and would spill at 3 or 4. Bounded proposals keep the half-width and the
// acceptance count live across the moves: their plain pass with 16-bit spins still fits 4 blocks
// per SM; the others run at 3, without spills.
// The tile of block b: a last tile column of at most 32 (64) columns runs as a 32- (64-) column
// tile of the same height (tile column 4 tx in 32-column units, 2 tx in 64-column units), as the
// batched kernels do: the energy partials, and so the energies, stay bit-identical between the
// two paths.
//
// Last wave (plain passes, a.nsplit > 0): the grid has nsplit blocks more than tiles; the last
// nsplit tiles run as two half-height tiles each (16 rows, blocks taken in pairs), so the final
// partial wave of blocks has twice as many, half as long: less of the machine idles while it
// drains. The host splits only when the half-lattice has no narrow last tile column and twice the
// remainder still fits one wave.
template <typename S, int R, bool MEASURE, int SAMPLE, bool PROP, int QM, bool HM, bool LATE>
__device__ __forceinline__ void block_tile(const SweepArgs& a, int b, TileSmem<R>& sm, void* eslot)
{
    const int ntx = (a.Lxh + kTJ - 1) / kTJ;
    if constexpr (!MEASURE && SAMPLE == 0) {
        if (a.nsplit > 0) {
            const int nfull = (int)gridDim.x - 2 * a.nsplit;   // tiles that run whole
            if (b >= nfull) {
                const int k = b - nfull, t = nfull + (k >> 1);
                sweep_tile<S, R / 2, false, 0, true, true, PROP, kTJ, QM, HM, LATE>(
                    a, t % ntx, 2 * (t / ntx) + (k & 1), *reinterpret_cast<TileSmem<R / 2>*>(&sm),
                    eslot);
                return;
            }
        }
    }
    const int tx = b % ntx, ty = b / ntx;
    const int rem = a.Lxh - tx * kTJ;
    if (tx == ntx - 1 && rem <= 32)
        sweep_tile<S, R / 4, MEASURE, SAMPLE, true, true, PROP, 32, QM, HM, LATE>(
            a, 4 * tx, ty, *reinterpret_cast<TileSmem<R / 4, 32>*>(&sm), eslot);
    else if (tx == ntx - 1 && rem <= 64)
        sweep_tile<S, R / 2, MEASURE, SAMPLE, true, true, PROP, 64, QM, HM, LATE>(
            a, 2 * tx, ty, *reinterpret_cast<TileSmem<R / 2, 64>*>(&sm), eslot);
    else
        sweep_tile<S, R, MEASURE, SAMPLE, true, true, PROP, kTJ, QM, HM, LATE>(a, tx, ty, sm, eslot);
}

template <typename S, int R, bool MEASURE, int SAMPLE, bool PROP, bool HM = false, bool LATE = false>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 2
                                       : ((PROP && (MEASURE || SAMPLE || sizeof(S) == 4)) ? 3 : 4))
    sweep_f32_kernel(const SweepArgs a)
{
    static_assert(R % 4 == 0, "the 64- and 32-column tail tiles have R / 2 and R / 4 rows per thread");
    __shared__ __align__(16) TileSmem<R> sm;
    // one tile per block, tiles row-major over a 1-D grid (no limit on the number of tile rows)
    const int b = blockIdx.x;
    void* eslot = nullptr;
    if (MEASURE)
        eslot = static_cast<char*>(a.epart) + (size_t)b * ((a.flags & kEnergyF32) ? 4 : 8);
    // the plain pass (most passes) with 16-bit spins has a copy for q = 1/2 (the paper's value
    // and the default) with q a compile-time constant; the branch is uniform over the grid (with
    // FP32 spins the second copy would spill registers)
    if constexpr (!MEASURE && SAMPLE == 0 && sizeof(S) == 2) {
        if (a.qf == 0.5f) {
            block_tile<S, R, MEASURE, SAMPLE, PROP, 2, HM, LATE>(a, b, sm, eslot);
            return;
        }
    }
    block_tile<S, R, MEASURE, SAMPLE, PROP, 0, HM, LATE>(a, b, sm, eslot);
}

// Launched as a programmatic dependent launch: while the previous pass's last blocks finish, this
// pass's blocks are scheduled and load their own rows (see sweep_tile).
template <typename S, bool MEASURE, int SAMPLE, bool PROP, bool HM = false>
cudaError_t go(const SweepArgs& a, cudaStream_t st)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(((a.Lxh + kTJ - 1) / kTJ) * ((a.Ly + tile_rows<kRows>() - 1) / tile_rows<kRows>())
                       + ((!MEASURE && SAMPLE == 0) ? a.nsplit : 0));
    cfg.blockDim = dim3(32, kWarps);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if constexpr (!MEASURE && SAMPLE == 0 && !PROP && sizeof(S) == 2) {
        if (a.late) return cudaLaunchKernelEx(&cfg, sweep_f32_kernel<S, kRows, false, 0, false, HM, true>, a);
    }
    return cudaLaunchKernelEx(&cfg, sweep_f32_kernel<S, kRows, MEASURE, SAMPLE, PROP, HM>, a);
}

template <typename S, bool PROP, bool HM = false>
cudaError_t dispatch_mode(const Precision& p, const SweepArgs& a, cudaStream_t st)
{
    const bool measure = (a.flags & kMeasure) && a.colour == 1;
    const int sample = (a.flags & kSample) ? (p.acc == 0 ? (a.part32 ? 3 : 1) : 2) : 0;
    if constexpr (sizeof(S) == 2) {   // fixed-point partial sums: FP16 spins only
        if (sample == 3)
            return measure ? go<S, true, 3, PROP, HM>(a, st) : go<S, false, 3, PROP, HM>(a, st);
    }
    if (sample == 3) return cudaErrorInvalidValue;
    if (measure) {
        if (sample == 0) return go<S, true, 0, PROP, HM>(a, st);
        if (sample == 1) return go<S, true, 1, PROP, HM>(a, st);
        return go<S, true, 2, PROP, HM>(a, st);
    }
    if (sample == 0) return go<S, false, 0, PROP, HM>(a, st);
    if (sample == 1) return go<S, false, 1, PROP, HM>(a, st);
    return go<S, false, 2, PROP, HM>(a, st);
}

template <bool PROP>
cudaError_t launch_store(const Precision& p, const SweepArgs& a, cudaStream_t st)
{
    if (p.func == 2) return cudaErrorInvalidValue;   // FP16 functions: launch_sweep_f32_half
    switch (p.store) {
    case kF64: return dispatch_mode<double, PROP>(p, a, st);
    case kF32: return dispatch_mode<float, PROP>(p, a, st);
    case kF16: return dispatch_mode<__half, PROP>(p, a, st);
    case kBF16: return dispatch_mode<__nv_bfloat16, PROP>(p, a, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace sweep_f32_detail
}  // namespace mpr
