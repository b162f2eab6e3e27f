// Newton-John kernels for GF(2^e), e = 9, 10 (template in nj_kernel.cuh).
#include "nj_kernel.cuh"

namespace m4rie {
template cudaError_t nj_launch<9>(const NjParams&, int, int64_t, int64_t, cudaStream_t);
template cudaError_t nj_launch<10>(const NjParams&, int, int64_t, int64_t, cudaStream_t);
}  // namespace m4rie
