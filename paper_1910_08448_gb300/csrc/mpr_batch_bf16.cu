// mpr_batch_bf16.cu -- the batched kernels for BF16 spin storage, every tile shape (one
// translation unit per storage type: the four compile in parallel).
#include "mpr_batch_kernels.cuh"

namespace mpr {
namespace batch {

Kernels kernels_bf16(int shape) { return table<__nv_bfloat16>(shape); }

}  // namespace batch
}  // namespace mpr
