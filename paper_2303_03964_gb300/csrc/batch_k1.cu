// batch_k1.cu -- the batch kernel for k = 1 (see batch_kernel.cuh); one file per k so
// that nvcc compiles the instantiations in parallel.
#include "batch_kernel.cuh"

namespace tfdp {
namespace bk {
TFDP_BATCH_INSTANTIATE(1)
}  // namespace bk
}  // namespace tfdp
