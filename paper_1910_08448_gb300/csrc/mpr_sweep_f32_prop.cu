// mpr_sweep_f32_prop.cu -- the FP32-function tile kernel (kind 0) with bounded Metropolis
// proposals of an adapted half-width (mpr_set_proposal); the kernel is in mpr_sweep_f32.cuh.
#include "mpr_sweep_f32.cuh"

namespace mpr {

cudaError_t launch_sweep_f32_prop(const Precision& p, const SweepArgs& a, cudaStream_t st)
{
    return sweep_f32_detail::launch_store<true>(p, a, st);
}

}  // namespace mpr
