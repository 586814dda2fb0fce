// mpr_sweep_f32_half.cu -- the tile kernel (kind 0) of the FP16-function setting X_F = H (FP16
// spins; the field's doubled angle in half2 arithmetic, atan2_doubled_h2 in mpr_tile_f32.cuh;
// everything else as in the FP32-function setting), uniform Metropolis proposals. Its own
// translation unit, so its instantiations compile in parallel with the others.
#include "mpr_sweep_f32.cuh"

namespace mpr {

cudaError_t launch_sweep_f32_half(const Precision& p, const SweepArgs& a, cudaStream_t st)
{
    if (p.store != kF16 || a.width) return cudaErrorInvalidValue;
    return sweep_f32_detail::dispatch_mode<__half, false, true>(p, a, st);
}

}  // namespace mpr
