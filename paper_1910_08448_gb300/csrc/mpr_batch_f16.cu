// mpr_batch_f16.cu -- the batched kernels for FP16 spin storage, every tile shape (one
// translation unit per storage type: the four compile in parallel).
#include "mpr_batch_kernels.cuh"

namespace mpr {
namespace batch {

Kernels kernels_f16(int shape) { return table<__half>(shape); }

}  // namespace batch
}  // namespace mpr
