// mpr_sweep_f32.cu -- single-problem colour half-sweep for the FP32 function setting: one launch
// per colour pass, one tile (mpr_tile_f32.cuh) per block.
#include "mpr_tile_f32.cuh"

namespace mpr {
namespace {

using namespace f32;

constexpr int kRows = 2;

template <typename S, int R, bool MEASURE, int SAMPLE>
__global__ void __launch_bounds__(256, 4) sweep_f32_kernel(const SweepArgs a)
{
    __shared__ __align__(16) TileSmem<R> sm;
    // one tile per block, tiles row-major over a 1-D grid (no limit on the number of tile rows)
    const int b = blockIdx.x;
    const int ntx = (a.Lxh + kTJ - 1) / kTJ;
    void* eslot = nullptr;
    if (MEASURE)
        eslot = static_cast<char*>(a.epart) + (size_t)b * ((a.flags & kEnergyF32) ? 4 : 8);
    sweep_tile<S, R, MEASURE, SAMPLE>(a, b % ntx, b / ntx, sm, eslot);
}

template <typename S, bool MEASURE, int SAMPLE>
cudaError_t go(const SweepArgs& a, cudaStream_t st)
{
    const dim3 grid(((a.Lxh + kTJ - 1) / kTJ) * ((a.Ly + tile_rows<kRows>() - 1) / tile_rows<kRows>()));
    sweep_f32_kernel<S, kRows, MEASURE, SAMPLE><<<grid, dim3(32, kWarps), 0, st>>>(a);
    return cudaGetLastError();
}

template <typename S>
cudaError_t dispatch_mode(const Precision& p, const SweepArgs& a, cudaStream_t st)
{
    const bool measure = (a.flags & kMeasure) && a.colour == 1;
    const int sample = (a.flags & kSample) ? (p.acc == 0 ? 1 : 2) : 0;
    if (measure) {
        if (sample == 0) return go<S, true, 0>(a, st);
        if (sample == 1) return go<S, true, 1>(a, st);
        return go<S, true, 2>(a, st);
    }
    if (sample == 0) return go<S, false, 0>(a, st);
    if (sample == 1) return go<S, false, 1>(a, st);
    return go<S, false, 2>(a, st);
}

}  // namespace

int sweep_f32_blocks(const Layout& L)
{
    return ((L.Lxh + kTJ - 1) / kTJ) * ((L.Ly + tile_rows<kRows>() - 1) / tile_rows<kRows>());
}

cudaError_t launch_sweep_f32(const Precision& p, const SweepArgs& a, cudaStream_t st)
{
    switch (p.store) {
    case kF64: return dispatch_mode<double>(p, a, st);
    case kF32: return dispatch_mode<float>(p, a, st);
    case kF16: return dispatch_mode<__half>(p, a, st);
    case kBF16: return dispatch_mode<__nv_bfloat16>(p, a, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace mpr
