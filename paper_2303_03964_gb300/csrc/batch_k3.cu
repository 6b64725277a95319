// batch_k3.cu -- the batch kernel for k = 3 (see batch_kernel.cuh); one file per k so
// that nvcc compiles the instantiations in parallel.
#include "batch_kernel.cuh"

namespace tfdp {
namespace bk {
TFDP_BATCH_INSTANTIATE(3)
}  // namespace bk
}  // namespace tfdp
