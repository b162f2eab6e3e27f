// Newton-John multiplication on packed rows (newton_john.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace m4rie {

// Section 3.1: bits per element in the packed representation (the next length
// dividing 64 that holds e bits).
__host__ __device__ constexpr int packed_width(int e) { return e <= 2 ? 2 : e <= 4 ? 4 : e <= 8 ? 8 : 16; }

struct NjParams {
  const void* A;  // m x k: elements (lda in elements) or packed rows (lda in 32-bit words)
  int64_t lda;
  const void* B;  // k x n, as A
  int64_t ldb;
  void* C;        // m x n, as A
  int64_t ldc;
  int64_t m, n, k;
  int packed;     // 1: A, B and C are packed rows; 0: element arrays
  int add;        // C += A B instead of C = A B
  uint32_t flow;  // f without its x^e term
  int* status;    // sticky device status word
  int vec_a, vec_b, vec_c;  // element rows of A / B / C start on 4-byte boundaries: 32-bit accesses allowed
  int vec16_b, vec16_c;    // element rows of B / C start on 16-byte boundaries: 16-byte accesses allowed
  int pdl;        // launch with programmatic dependent launch
  // filled by launch_newton_john from the plan
  int64_t nw;     // 32-bit words per packed row of B and C
  int lg;         // log2 of the tile width in words
  int ks;         // CTAs per cluster, each over its own k range
  int64_t kper;   // rows of k per cluster rank
};

struct NjPlan {
  int lg, R, ks;
  int64_t tiles_m, tiles_n, kper, nw;
};

template <int E>
cudaError_t nj_launch(const NjParams& p, int R, int64_t tiles_m, int64_t tiles_n, cudaStream_t s);

NjPlan plan_newton_john(int e, int64_t m, int64_t n, int64_t k, bool packed, int num_sms);
cudaError_t launch_newton_john(int e, const NjParams& p, const NjPlan& plan, cudaStream_t s, int64_t* launches);

// Element arrays (row stride ldx elements) <-> packed rows (ld32 words of 32
// bits per row).  to_packed zeroes padding and flags entries >= 2^e.
cudaError_t launch_to_packed(int e, int64_t rows, int64_t cols, const void* X, int64_t ldx, uint32_t* out,
                             int64_t ld32, int* status, cudaStream_t s, int64_t* launches);
cudaError_t launch_from_packed(int e, int64_t rows, int64_t cols, const uint32_t* in, int64_t ld32, void* X,
                               int64_t ldx, cudaStream_t s, int64_t* launches);

}  // namespace m4rie
