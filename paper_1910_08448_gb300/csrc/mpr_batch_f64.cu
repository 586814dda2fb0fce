// mpr_batch_f64.cu -- the batched kernels for FP64 spin storage, every tile shape (one
// translation unit per storage type: the four compile in parallel).
#include "mpr_batch_kernels.cuh"

namespace mpr {
namespace batch {

Kernels kernels_f64(int shape) { return table<double>(shape); }

}  // namespace batch
}  // namespace mpr
