// Slicing kernels (Section 3.2, Figure 1) and the GEMM operand planes built from them.
//
// Every operand plane entry is parity(x & mask) of one element x: the slice
// A_j is the mask 1 << j, a Karatsuba operand sum (A_0 + A_1, Section 5) is the
// mask 0b11, and the slice (alpha^j B)_i of the scaled matrix of Algorithm 2 is
// the mask whose bit l is coefficient i of x^(j+l) mod f.  So one kernel per
// layout serves every schedule.  All kernels are HBM-bound; loads are
// coalesced along rows and bits are gathered with warp ballots.
#include "m4rie_internal.cuh"

namespace m4rie {
namespace {

__device__ __forceinline__ uint32_t par(uint32_t x) { return __popc(x) & 1u; }

__device__ __forceinline__ int64_t plane_index(const PackParams& p, int q, int64_t r, int64_t t) {
  const int per_b = p.nb * p.kb;
  const int b = q / per_b;
  const int i = (q / p.kb) % p.nb;
  const int j = q % p.kb;
  const int64_t G = p.G;
  const int64_t orow = (r / G) * p.nb * G + (int64_t)i * G + (r % G);
  return (int64_t)b * p.bstride + orow * p.ld + (int64_t)j * p.Kp + t;
}

template <typename T>
__device__ __forceinline__ uint32_t load_elem(const PackParams& p, int64_t r, int64_t c) {
  return (uint32_t)static_cast<const T*>(p.X)[r * p.ldx + c];
}

__device__ __forceinline__ void flag_range(int* status, bool bad) {
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusRange);
}

// ---- A side, byte / nibble planes: one thread per (row, 16 consecutive t).
template <typename T, bool NIB>
__global__ void pack_rows_bytes(const __grid_constant__ PackParams p) {
  const int64_t nch = p.Kp / 16;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = idx < p.rows_p * nch;
  const int64_t r = live ? idx / nch : 0;
  const int64_t t0 = live ? (idx % nch) * 16 : 0;
  uint32_t x[16];
  bool bad = false;
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int64_t t = t0 + u;
    x[u] = (live && r < p.rows && t < p.K) ? load_elem<T>(p, r, t) : 0u;
    bad |= x[u] > p.emask;
    x[u] &= p.emask;
  }
  flag_range(p.status, bad);
  if (!live) return;
  for (int q = 0; q < p.P; ++q) {
    const uint32_t mk = p.mask[q];
    const int64_t o = plane_index(p, q, r, t0);
    if (!NIB) {
      uint32_t w[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        w[k] = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) w[k] |= (par(x[4 * k + u] & mk) * p.one) << (8 * u);
      }
      *reinterpret_cast<uint4*>(static_cast<uint8_t*>(p.out) + o) = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
      uint32_t w[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        w[k] = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) w[k] |= (par(x[8 * k + u] & mk) * p.one) << (4 * u);
      }
      *reinterpret_cast<uint2*>(static_cast<uint8_t*>(p.out) + o / 2) = make_uint2(w[0], w[1]);
    }
  }
}

// ---- A side, bit planes: one warp per (row, 512 consecutive t).  Lanes load
// 16 consecutive elements each, stage them in shared memory, and every
// output word is one ballot over 32 consecutive elements.
template <typename T>
__global__ void __launch_bounds__(256) pack_rows_bits(const __grid_constant__ PackParams p) {
  __shared__ uint32_t sx[8][512];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nch = (p.Kp + 511) / 512;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const bool live = wid < p.rows_p * nch;  // warp-uniform
  const int64_t r = live ? wid / nch : 0;
  const int64_t tb = live ? (wid % nch) * 512 : 0;
  bool bad = false;
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int64_t t = tb + 16 * lane + u;
    uint32_t v = (live && r < p.rows && t < p.K) ? load_elem<T>(p, r, t) : 0u;
    bad |= v > p.emask;
    sx[wib][16 * lane + u] = v & p.emask;
  }
  flag_range(p.status, bad);
  __syncwarp();
  if (!live) return;
  uint32_t x[16];
#pragma unroll
  for (int w = 0; w < 16; ++w) x[w] = sx[wib][32 * w + lane];
  const bool store = tb + 32 * lane < p.Kp && lane < 16;
  for (int q = 0; q < p.P; ++q) {
    const uint32_t mk = p.mask[q];
    uint32_t my = 0;
#pragma unroll
    for (int w = 0; w < 16; ++w) {
      const uint32_t wd = __ballot_sync(0xffffffffu, par(x[w] & mk));
      my = (lane == w) ? wd : my;
    }
    if (store) static_cast<uint32_t*>(p.out)[plane_index(p, q, r, tb) / 32 + lane] = my;
  }
}

// ---- B side (columns of X become plane rows), byte / nibble planes.
// Tile of 64 t x 64 columns staged in shared memory (one 32-bit word per
// element, conflict-free column reads); one thread per (column, 16 t).
template <typename T, bool NIB>
__global__ void __launch_bounds__(256) pack_cols_bytes(const __grid_constant__ PackParams p) {
  __shared__ uint32_t tile[64][65];
  const int64_t c0 = (int64_t)blockIdx.x * 64, t0 = (int64_t)blockIdx.y * 64;
  bool bad = false;
  for (int idx = threadIdx.x; idx < 64 * 64; idx += 256) {
    const int tt = idx >> 6, cc = idx & 63;
    const int64_t t = t0 + tt, c = c0 + cc;
    uint32_t v = (t < p.K && c < p.rows) ? (uint32_t) static_cast<const T*>(p.X)[t * p.ldx + c] : 0u;
    bad |= v > p.emask;
    tile[tt][cc] = v & p.emask;
  }
  flag_range(p.status, bad);
  __syncthreads();
  const int cl = threadIdx.x >> 2, ch = threadIdx.x & 3;
  const int64_t c = c0 + cl;
  if (c >= p.rows_p) return;
  uint32_t x[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) x[u] = tile[ch * 16 + u][cl];
  const int64_t tt0 = t0 + ch * 16;
  for (int q = 0; q < p.P; ++q) {
    const uint32_t mk = p.mask[q];
    const int64_t o = plane_index(p, q, c, tt0);
    if (!NIB) {
      uint32_t w[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        w[k] = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) w[k] |= (par(x[4 * k + u] & mk) * p.one) << (8 * u);
      }
      *reinterpret_cast<uint4*>(static_cast<uint8_t*>(p.out) + o) = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
      uint32_t w[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        w[k] = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) w[k] |= (par(x[8 * k + u] & mk) * p.one) << (4 * u);
      }
      *reinterpret_cast<uint2*>(static_cast<uint8_t*>(p.out) + o / 2) = make_uint2(w[0], w[1]);
    }
  }
}

// ---- B side, bit planes: tile of 128 t x 64 columns; each warp owns 8
// columns; lane l reads t = 32 s + l, one ballot per (mask, s) gives a word.
template <typename T>
__global__ void __launch_bounds__(256) pack_cols_bits(const __grid_constant__ PackParams p) {
  __shared__ uint32_t tile[128][65];
  const int64_t c0 = (int64_t)blockIdx.x * 64, t0 = (int64_t)blockIdx.y * 128;
  bool bad = false;
  for (int idx = threadIdx.x; idx < 128 * 64; idx += 256) {
    const int tt = idx >> 6, cc = idx & 63;
    const int64_t t = t0 + tt, c = c0 + cc;
    uint32_t v = (t < p.K && c < p.rows) ? (uint32_t) static_cast<const T*>(p.X)[t * p.ldx + c] : 0u;
    bad |= v > p.emask;
    tile[tt][cc] = v & p.emask;
  }
  flag_range(p.status, bad);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int cc = 0; cc < 8; ++cc) {
    const int cl = w * 8 + cc;
    const int64_t c = c0 + cl;
    if (c >= p.rows_p) break;  // warp-uniform
    uint32_t x[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) x[s] = tile[32 * s + lane][cl];
    for (int q0 = 0; q0 < p.P; q0 += 32) {
      const int cnt = min(32, p.P - q0);
      uint32_t my[4] = {0, 0, 0, 0};
      for (int qq = 0; qq < cnt; ++qq) {
        const uint32_t mk = p.mask[q0 + qq];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const uint32_t wd = __ballot_sync(0xffffffffu, par(x[s] & mk));
          my[s] = (lane == qq) ? wd : my[s];
        }
      }
      if (lane < cnt) {
        uint32_t* o = static_cast<uint32_t*>(p.out) + plane_index(p, q0 + lane, c, t0) / 32;
        *reinterpret_cast<uint4*>(o) = make_uint4(my[0], my[1], my[2], my[3]);
      }
    }
  }
}

// ---- Public slice format: one warp per (row, 64-bit word).
template <typename T>
__global__ void __launch_bounds__(256) slice_kernel(int e, int64_t rows, int64_t cols, const T* __restrict__ X,
                                                    uint64_t* __restrict__ S, int64_t ldw, int* status) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const bool live = wid < rows * ldw;
  const int64_t r = live ? wid / ldw : 0, w = live ? wid % ldw : 0;
  const uint32_t emask = (1u << e) - 1;
  const int64_t c_lo = 64 * w + lane, c_hi = c_lo + 32;
  uint32_t x0 = (live && c_lo < cols) ? (uint32_t)X[r * cols + c_lo] : 0u;
  uint32_t x1 = (live && c_hi < cols) ? (uint32_t)X[r * cols + c_hi] : 0u;
  flag_range(status, (x0 | x1) > emask);
  if (!live) return;
  uint64_t mine = 0;
  for (int i = 0; i < e; ++i) {
    const uint32_t lo = __ballot_sync(0xffffffffu, (x0 >> i) & 1u);
    const uint32_t hi = __ballot_sync(0xffffffffu, (x1 >> i) & 1u);
    if (lane == i) mine = (uint64_t)lo | ((uint64_t)hi << 32);
  }
  if (lane < e) S[((int64_t)lane * rows + r) * ldw + w] = mine;
}

// ---- Clinging: one warp per (row, word); lane l writes columns 64w+l and 64w+32+l.
template <typename T>
__global__ void __launch_bounds__(256) cling_kernel(int e, int64_t rows, int64_t cols, const uint64_t* __restrict__ S,
                                                    int64_t ldw, T* __restrict__ X) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (cols + 63) / 64;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (wid >= rows * nw) return;
  const int64_t r = wid / nw, w = wid % nw;
  uint32_t v0 = 0, v1 = 0;
  for (int i = 0; i < e; ++i) {
    const uint64_t word = S[((int64_t)i * rows + r) * ldw + w];
    v0 |= (uint32_t)((word >> lane) & 1u) << i;
    v1 |= (uint32_t)((word >> (lane + 32)) & 1u) << i;
  }
  const int64_t c_lo = 64 * w + lane, c_hi = c_lo + 32;
  if (c_lo < cols) X[r * cols + c_lo] = (T)v0;
  if (c_hi < cols) X[r * cols + c_hi] = (T)v1;
}

// ---- Karatsuba recombination: bit s of C[r][c] is the parity of the
// products selected by out_mask[s] (reduction mod f folded in).
template <typename T>
__global__ void __launch_bounds__(256) recombine_kernel(const __grid_constant__ RecombineParams p) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = idx < p.m * p.n;
  const int64_t r = live ? idx / p.n : 0, c = live ? idx % p.n : 0;
  uint64_t v = 0;
  if (live)
    for (int q = 0; q < p.r; ++q) {
      const uint32_t w = p.P[((int64_t)q * p.rows_p + r) * p.ldw + (c >> 5)];
      v |= (uint64_t)((w >> (c & 31)) & 1u) << q;
    }
  uint32_t out = 0;
  for (int s = 0; s < p.e; ++s) out |= (uint32_t)(__popcll(v & p.out_mask[s]) & 1) << s;
  bool bad = false;
  T* C = static_cast<T*>(p.C);
  if (live && p.add) {
    uint32_t old = (uint32_t)C[r * p.ldc + c];
    bad = old > p.emask;
    out ^= old & p.emask;
  }
  flag_range(p.status, bad);
  if (live) C[r * p.ldc + c] = (T)out;
}

template <typename K, typename... Args>
cudaError_t launch(K kernel, int64_t blocks, int threads, cudaStream_t s, int64_t* launches, Args... args) {
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  kernel<<<(unsigned)blocks, threads, 0, s>>>(args...);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pack_planes(const PackParams& p, bool trans, cudaStream_t s, int64_t* launches) {
  const bool u16 = p.elem_bytes == 2;
  if (!trans) {
    if (p.fmt == kFmtBit) {
      const int64_t warps = p.rows_p * ((p.Kp + 511) / 512);
      return u16 ? launch(pack_rows_bits<uint16_t>, ceil_div(warps, 8), 256, s, launches, p)
                 : launch(pack_rows_bits<uint8_t>, ceil_div(warps, 8), 256, s, launches, p);
    }
    const int64_t threads = p.rows_p * (p.Kp / 16);
    if (p.fmt == kFmtByte)
      return u16 ? launch(pack_rows_bytes<uint16_t, false>, ceil_div(threads, 256), 256, s, launches, p)
                 : launch(pack_rows_bytes<uint8_t, false>, ceil_div(threads, 256), 256, s, launches, p);
    return u16 ? launch(pack_rows_bytes<uint16_t, true>, ceil_div(threads, 256), 256, s, launches, p)
               : launch(pack_rows_bytes<uint8_t, true>, ceil_div(threads, 256), 256, s, launches, p);
  }
  const int64_t gx = ceil_div(p.rows_p, 64);
  if (gx > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (p.fmt == kFmtBit) {
    const int64_t gy = p.Kp / 128;
    if (gy > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)gx, (unsigned)gy);
    if (u16) pack_cols_bits<uint16_t><<<grid, 256, 0, s>>>(p);
    else pack_cols_bits<uint8_t><<<grid, 256, 0, s>>>(p);
  } else {
    const int64_t gy = p.Kp / 64;
    if (gy > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)gx, (unsigned)gy);
    if (p.fmt == kFmtByte) {
      if (u16) pack_cols_bytes<uint16_t, false><<<grid, 256, 0, s>>>(p);
      else pack_cols_bytes<uint8_t, false><<<grid, 256, 0, s>>>(p);
    } else {
      if (u16) pack_cols_bytes<uint16_t, true><<<grid, 256, 0, s>>>(p);
      else pack_cols_bytes<uint8_t, true><<<grid, 256, 0, s>>>(p);
    }
  }
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_slice(int e, int64_t rows, int64_t cols, const void* elems, uint64_t* slices, int64_t ld_words,
                         int* status, cudaStream_t s, int64_t* launches) {
  const int64_t warps = rows * ld_words;
  if (e > 8)
    return launch(slice_kernel<uint16_t>, ceil_div(warps, 8), 256, s, launches, e, rows, cols,
                  static_cast<const uint16_t*>(elems), slices, ld_words, status);
  return launch(slice_kernel<uint8_t>, ceil_div(warps, 8), 256, s, launches, e, rows, cols,
                static_cast<const uint8_t*>(elems), slices, ld_words, status);
}

cudaError_t launch_cling(int e, int64_t rows, int64_t cols, const uint64_t* slices, int64_t ld_words, void* elems,
                         cudaStream_t s, int64_t* launches) {
  const int64_t warps = rows * ceil_div(cols, 64);
  if (e > 8)
    return launch(cling_kernel<uint16_t>, ceil_div(warps, 8), 256, s, launches, e, rows, cols, slices, ld_words,
                  static_cast<uint16_t*>(elems));
  return launch(cling_kernel<uint8_t>, ceil_div(warps, 8), 256, s, launches, e, rows, cols, slices, ld_words,
                static_cast<uint8_t*>(elems));
}

cudaError_t launch_recombine(const RecombineParams& p, cudaStream_t s, int64_t* launches) {
  const int64_t n = p.m * p.n;
  if (p.elem_bytes == 2) return launch(recombine_kernel<uint16_t>, ceil_div(n, 256), 256, s, launches, p);
  return launch(recombine_kernel<uint8_t>, ceil_div(n, 256), 256, s, launches, p);
}

}  // namespace m4rie
