// mpr_sweep_f32.cu -- the FP32-function tile kernel (kind 0) with uniform Metropolis proposals,
// and the entry point that picks the uniform or the bounded-proposal variants
// (mpr_sweep_f32_prop.cu). The kernel itself is in mpr_sweep_f32.cuh.
#include "mpr_sweep_f32.cuh"

namespace mpr {

int sweep_f32_blocks(const Layout& L)
{
    using namespace sweep_f32_detail;
    return ((L.Lxh + kTJ - 1) / kTJ) * ((L.Ly + tile_rows<kRows>() - 1) / tile_rows<kRows>());
}

int sweep_f32_plain_occupancy(const Precision& p)
{
    using namespace sweep_f32_detail;
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (p.store) {
    case kF64:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_f32_kernel<double, kRows, false, 0, false>, 256, 0);
        break;
    case kF32:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_f32_kernel<float, kRows, false, 0, false>, 256, 0);
        break;
    case kF16:
        // (the FP16-function variant has the same launch bounds and shared memory)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_f32_kernel<__half, kRows, false, 0, false>, 256, 0);
        break;
    case kBF16:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_f32_kernel<__nv_bfloat16, kRows, false, 0, false>, 256, 0);
        break;
    default: break;
    }
    return e == cudaSuccess ? n : 0;
}

cudaError_t launch_sweep_f32(const Precision& p, const SweepArgs& a, cudaStream_t st)
{
    if (p.func == 2) return launch_sweep_f32_half(p, a, st);
    if (a.width) return launch_sweep_f32_prop(p, a, st);
    return sweep_f32_detail::launch_store<false>(p, a, st);
}

}  // namespace mpr
