// batch_k2.cu -- the batch kernel for k = 2 (see batch_kernel.cuh); one file per k so
// that nvcc compiles the instantiations in parallel.
#include "batch_kernel.cuh"

namespace tfdp {
namespace bk {
TFDP_BATCH_INSTANTIATE(2)
}  // namespace bk
}  // namespace tfdp
