// Row moves shared by the echelon form and the PLE decomposition
// (echelon.cu, ple.cu): rows src[j] -> dst[j] of a row-major matrix, columns
// c0 .. c0 + nt - 1, through a scratch buffer (gather, then scatter), the
// index lists staged in pinned host memory.
#pragma once
#include <algorithm>
#include <vector>

#include "context.h"

namespace m4rie {
namespace rowmove {

constexpr int kRows = 96;               // rows per move list, at most (one candidate block)
constexpr int kSlot = 4 * kRows;        // ints per pinned slot: up to 2 kRows (src, dst) pairs

struct Bufs {
  int* moves = nullptr;     // device: two slots of [src | dst]
  int* host = nullptr;      // pinned: two slots of [src | dst]
  uint8_t* tmp = nullptr;   // device: 2 kRows rows of the moved width
};

inline size_t elem_bytes(int e) { return e <= 8 ? 1 : 2; }

inline m4rie_status fail(m4rie_ctx* ctx, cudaError_t err) {
  ctx->last_error = cudaGetErrorString(err);
  return M4RIE_ERR_CUDA;
}

// The look-ahead side stream of the echelon form and the PLE decomposition
// (created at the highest priority, so that a panel kernel queued on it is
// dispatched ahead of the products queued on the main stream), its two
// events and the pinned pivot list.
inline cudaError_t ensure_side(m4rie_ctx* ctx) {
  if (ctx->ech_side) return cudaSuccess;
  int lo = 0, hi = 0;
  cudaError_t err = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (err != cudaSuccess) return err;
  if ((err = cudaStreamCreateWithPriority(&ctx->ech_side, cudaStreamNonBlocking, hi)) != cudaSuccess ||
      (err = cudaEventCreateWithFlags(&ctx->ech_ev[0], cudaEventDisableTiming)) != cudaSuccess ||
      (err = cudaEventCreateWithFlags(&ctx->ech_ev[1], cudaEventDisableTiming)) != cudaSuccess ||
      (err = cudaMallocHost(&ctx->ech_po_host, kPanelHostBytes)) != cudaSuccess)
    return err;
  return cudaSuccess;
}

template <typename T>
__global__ void gather_rows(const T* __restrict__ A, int64_t lda, int64_t c0, int64_t nt, const int* __restrict__ src,
                            T* __restrict__ tmp) {
  const int j = blockIdx.y;
  const T* s = A + (int64_t)src[j] * lda + c0;
  T* d = tmp + (int64_t)j * nt;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nt; c += (int64_t)gridDim.x * blockDim.x)
    d[c] = s[c];
}

template <typename T>
__global__ void scatter_rows(T* __restrict__ A, int64_t lda, int64_t c0, int64_t nt, const int* __restrict__ dst,
                             const T* __restrict__ tmp) {
  const int j = blockIdx.y;
  T* d = A + (int64_t)dst[j] * lda + c0;
  const T* s = tmp + (int64_t)j * nt;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nt; c += (int64_t)gridDim.x * blockDim.x)
    d[c] = s[c];
}

// At most 2 kRows moves, staged in pinned slot `slot`.  A slot is written
// again only after a later read-back has synchronized the stream, so no wait
// is needed here.
template <typename T>
cudaError_t move_rows(m4rie_ctx* ctx, const Bufs& w, int slot, T* A, int64_t lda, int64_t c0, int64_t nt,
                      const std::vector<int>& src, const std::vector<int>& dst) {
  const int nm = (int)src.size();
  if (nm == 0 || nt == 0) return cudaSuccess;
  if (nm > 2 * kRows) return cudaErrorInvalidValue;
  int* h = w.host + slot * kSlot;
  int* d = w.moves + slot * kSlot;
  std::copy(src.begin(), src.end(), h);
  std::copy(dst.begin(), dst.end(), h + nm);
  cudaError_t err = cudaMemcpyAsync(d, h, sizeof(int) * 2 * nm, cudaMemcpyHostToDevice, ctx->stream);
  if (err != cudaSuccess) return err;
  const dim3 grid((unsigned)std::min<int64_t>(ceil_div(nt, 256), 64), (unsigned)nm);
  gather_rows<T><<<grid, 256, 0, ctx->stream>>>(A, lda, c0, nt, d, reinterpret_cast<T*>(w.tmp));
  scatter_rows<T><<<grid, 256, 0, ctx->stream>>>(A, lda, c0, nt, d + nm, reinterpret_cast<const T*>(w.tmp));
  ctx->launches += 2;
  return cudaGetLastError();
}

}  // namespace rowmove
}  // namespace m4rie
