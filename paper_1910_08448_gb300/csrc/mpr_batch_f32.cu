// mpr_batch_f32.cu -- the batched kernels for FP32 spin storage, every tile shape (one
// translation unit per storage type: the four compile in parallel).
#include "mpr_batch_kernels.cuh"

namespace mpr {
namespace batch {

Kernels kernels_f32(int shape) { return table<float>(shape); }

}  // namespace batch
}  // namespace mpr
