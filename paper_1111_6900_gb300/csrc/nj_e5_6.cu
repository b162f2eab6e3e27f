// Newton-John kernels for GF(2^e), e = 5, 6 (template in nj_kernel.cuh).
#include "nj_kernel.cuh"

namespace m4rie {
template cudaError_t nj_launch<5>(const NjParams&, int, int64_t, int64_t, cudaStream_t);
template cudaError_t nj_launch<6>(const NjParams&, int, int64_t, int64_t, cudaStream_t);
}  // namespace m4rie
