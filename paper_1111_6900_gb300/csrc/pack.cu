// Slicing kernels (Section 3.2, Figure 1) and the GEMM operand planes built from them.
//
// Every operand plane entry is parity(x & mask) of one element x: the slice
// A_j is the mask 1 << j, a Karatsuba operand sum (A_0 + A_1, Section 5) is the
// mask 0b11, and the slice (alpha^j B)_i of the scaled matrix of Algorithm 2 is
// the mask whose bit l is coefficient i of x^(j+l) mod f.  So one kernel per
// layout serves every schedule.  All kernels are HBM-bound; loads are
// coalesced along rows and bits are gathered with warp ballots.
#include <algorithm>

#include "m4rie_internal.cuh"

namespace m4rie {
namespace {

__device__ __forceinline__ uint32_t par(uint32_t x) { return __popc(x) & 1u; }

// Plane addressing: entry (q, r, t) is at qoff[q] + row_offset(r) + t with
// qoff[q] = b*bstride + i*G*ld + j*Kp  (q = (b*nb + i)*kb + j) and
// row_offset(r) = ((r / G) * nb * G + r % G) * ld.  qoff is computed once per
// block into shared memory so the per-entry work has no divisions.
__device__ __forceinline__ void fill_qoff(const PackParams& p, int64_t* qoff) {
  for (int q = threadIdx.x; q < p.P; q += blockDim.x) {
    const int b = q / (p.nb * p.kb), i = (q / p.kb) % p.nb, j = q % p.kb;
    qoff[q] = (int64_t)b * p.bstride + (int64_t)i * p.G * p.ld + (int64_t)j * p.Kp;
  }
}
__device__ __forceinline__ int64_t row_offset(const PackParams& p, int64_t r) {
  // r < 2^31 and G < 2^16 (validated on the host): 32-bit division
  const uint32_t rr = (uint32_t)r, G = (uint32_t)p.G;
  const uint32_t g = rr / G;
  return ((int64_t)g * p.nb * G + (rr - g * G)) * p.ld;
}

// Warp-wide lookup of XOR combinations of the slice words: after
// build_xor_table, lane l holds lo = XOR of S[b] over the bits b < 5 of l and
// hi = XOR of S[5 + b] over the bits b of l; the combination for any mask is
// then two shuffles and one XOR.
struct XorTable {
  uint32_t lo, hi;
};
__device__ __forceinline__ XorTable build_xor_table(const uint32_t (&S)[10], int e, int lane) {
  XorTable t{0, 0};
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    if (b < e && (lane >> b & 1)) t.lo ^= S[b];
    if (b + 5 < e && (lane >> b & 1)) t.hi ^= S[b + 5];
  }
  return t;
}
__device__ __forceinline__ uint32_t xor_lookup(const XorTable& t, uint32_t mask, int e) {
  uint32_t w = __shfl_sync(0xffffffffu, t.lo, mask & 31u);
  if (e > 5) w ^= __shfl_sync(0xffffffffu, t.hi, (mask >> 5) & 31u);
  return w;
}

template <typename T>
__device__ __forceinline__ uint32_t load_elem(const PackParams& p, int64_t r, int64_t c) {
  return (uint32_t)static_cast<const T*>(p.X)[r * p.ldx + c];
}

__device__ __forceinline__ void flag_range(int* status, bool bad) {
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusRange);
}

// ---- Slice words.  Bit u of slice word l is coefficient l of element u; an
// operand plane for mask q is the XOR of the slice words selected by q.

// 16 consecutive elements of row r starting at t0 (zeros past the row end),
// as 4 words of bytes (u8) or 8 words of halfwords (u16).
template <typename T>
__device__ __forceinline__ void load16(const PackParams& p, int64_t r, int64_t t0, uint32_t (&v)[8]) {
  const T* row = static_cast<const T*>(p.X) + r * p.ldx;
  constexpr int W = sizeof(T) == 1 ? 4 : 8;
  if (p.vec && t0 + 16 <= p.K) {
    const uint4* q = reinterpret_cast<const uint4*>(row + t0);
    const uint4 a = q[0];
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
    if (W == 8) {
      const uint4 b = q[1];
      v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < W; ++k) v[k] = 0;
#pragma unroll
    for (int u = 0; u < 16; ++u)
      if (t0 + u < p.K) v[u * sizeof(T) / 4] |= (uint32_t)row[t0 + u] << (8 * sizeof(T) * (u % (4 / sizeof(T))));
  }
}

// Range check and masking of packed elements; returns true if any was >= 2^e.
template <typename T>
__device__ __forceinline__ bool clamp16(uint32_t (&v)[8], uint32_t emask) {
  constexpr int W = sizeof(T) == 1 ? 4 : 8;
  const uint32_t rep = sizeof(T) == 1 ? emask * 0x01010101u : emask * 0x00010001u;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    bad |= (v[k] & ~rep) != 0;
    v[k] &= rep;
  }
  return bad;
}

// Slice words of 16 packed elements: S[l] bit u = bit l of element u.
template <typename T>
__device__ __forceinline__ void slices16(const uint32_t (&v)[8], int e, uint32_t (&S)[10]) {
#pragma unroll
  for (int l = 0; l < 10; ++l) {
    uint32_t w = 0;
    if (l < e) {
      if (sizeof(T) == 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) w |= ((((v[k] >> l) & 0x01010101u) * 0x01020408u) >> 24) << (4 * k);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) w |= (((((v[k] >> l) & 0x00010001u) * 0x00008001u) >> 15) & 3u) << (2 * k);
      }
    }
    S[l] = w;
  }
}

__device__ __forceinline__ uint32_t combine(const uint32_t (&S)[10], int e, uint32_t mask) {
  uint32_t w = 0;
#pragma unroll
  for (int l = 0; l < 10; ++l)
    if (l < e && (mask >> l & 1u)) w ^= S[l];
  return w;
}

// 16 plane bits -> 16 bytes (0 or `one`) or 16 nibbles.
__device__ __forceinline__ void store_bytes16(uint8_t* dst, uint32_t bits, uint32_t one) {
  uint32_t w[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) w[k] = (((bits >> (4 * k)) & 0xFu) * 0x00204081u & 0x01010101u) * one;
  *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ void store_nibs16(uint8_t* dst, uint32_t bits, uint32_t one) {
  uint32_t w[2] = {0, 0};
#pragma unroll
  for (int u = 0; u < 16; ++u) w[u >> 3] |= ((bits >> u) & 1u) * one << (4 * (u & 7));
  *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
}

// ---- A side, byte / nibble planes: one thread per (row, 16 consecutive t).
// grid.x covers the 16-element chunks of a row, grid.y strides over rows.
template <typename T, bool NIB>
__global__ void __launch_bounds__(256) pack_rows_bytes(const __grid_constant__ PackParams p) {
  __shared__ int64_t qoff[kMaxMasks];
  fill_qoff(p, qoff);
  __syncthreads();
  const int64_t t0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 16;
  const bool live_t = t0 < p.Kp;
  uint8_t* out = static_cast<uint8_t*>(p.out);
  for (int64_t r = blockIdx.y; r < p.rows_p; r += gridDim.y) {
    uint32_t v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (live_t && r < p.rows) load16<T>(p, r, t0, v);
    flag_range(p.status, clamp16<T>(v, p.emask));
    if (!live_t) continue;
    uint32_t S[10];
    slices16<T>(v, p.e, S);
    const int64_t base = row_offset(p, r) + t0;
    for (int q = 0; q < p.P; ++q) {
      const uint32_t bits = combine(S, p.e, p.mask[q]);
      const int64_t o = qoff[q] + base;
      if (NIB) store_nibs16(out + o / 2, bits, p.one);
      else store_bytes16(out + o, bits, p.one);
    }
  }
}

// ---- A side, bit planes: one warp per (row, 512 consecutive t).  Lane l
// holds t = 16 l .. 16 l + 15; lane pairs form 32-bit words.
// grid.x * 8 warps cover the 512-element chunks of a row, grid.y strides over rows.
template <typename T>
__global__ void __launch_bounds__(256) pack_rows_bits(const __grid_constant__ PackParams p) {
  __shared__ int64_t qoff[kMaxMasks];
  fill_qoff(p, qoff);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t tb = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * 512;
  const bool live_t = tb < p.Kp;  // warp-uniform
  uint32_t* out = static_cast<uint32_t*>(p.out);
  for (int64_t r = blockIdx.y; r < p.rows_p; r += gridDim.y) {
    uint32_t v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (live_t && r < p.rows) load16<T>(p, r, tb + 16 * lane, v);
    flag_range(p.status, clamp16<T>(v, p.emask));
    if (!live_t) continue;
    uint32_t S[10];
    slices16<T>(v, p.e, S);
#pragma unroll
    for (int l = 0; l < 10; ++l) S[l] |= __shfl_down_sync(0xffffffffu, S[l], 1) << 16;
    // lanes 2w now hold word w of every slice; share the XOR table of those words
    const bool store = (lane & 1) == 0 && tb + 16 * lane < p.Kp;
    const int64_t base = (row_offset(p, r) + tb) / 32 + (lane >> 1);
    for (int q = 0; q < p.P; ++q) {
      const uint32_t w = combine(S, p.e, p.mask[q]);
      if (store) out[qoff[q] / 32 + base] = w;
    }
  }
}

// Stage a tile of TT rows (t) x 64 columns of X into shared memory, one
// 32-bit word per element; masks the elements and reports out-of-range ones.
template <typename T, int TT>
__device__ __forceinline__ void stage_tile(const PackParams& p, int64_t t0, int64_t c0, uint32_t (*tile)[65]) {
  bool bad = false;
  const T* X = static_cast<const T*>(p.X);
  constexpr int CH = 64 * sizeof(T) / 16;  // 16-byte chunks per tile row
  if (p.vec && c0 + 64 <= p.rows && t0 + TT <= p.K) {
    for (int idx = threadIdx.x; idx < TT * CH; idx += blockDim.x) {
      const int tt = idx / CH, ch = idx % CH;
      const uint4 a = *reinterpret_cast<const uint4*>(X + (t0 + tt) * p.ldx + c0 + ch * (16 / sizeof(T)));
      const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int k = 0; k < 16 / (int)sizeof(T); ++k) {
        const uint32_t x = sizeof(T) == 1 ? (w[k >> 2] >> (8 * (k & 3))) & 0xFFu : (w[k >> 1] >> (16 * (k & 1))) & 0xFFFFu;
        bad |= x > p.emask;
        tile[tt][ch * (16 / sizeof(T)) + k] = x & p.emask;
      }
    }
  } else {
    for (int idx = threadIdx.x; idx < TT * 64; idx += blockDim.x) {
      const int tt = idx >> 6, cc = idx & 63;
      const int64_t t = t0 + tt, c = c0 + cc;
      const uint32_t x = (t < p.K && c < p.rows) ? (uint32_t)X[t * p.ldx + c] : 0u;
      bad |= x > p.emask;
      tile[tt][cc] = x & p.emask;
    }
  }
  flag_range(p.status, bad);
}

// ---- B side (columns of X become plane rows), bit planes.  Tile of 128 t x
// 64 columns; each warp owns 8 columns; lane l reads t = 32 s + l; e ballots
// per 32 elements give the slice words, lane q forms plane q by XORs.
template <typename T>
__global__ void __launch_bounds__(256) pack_cols_bits(const __grid_constant__ PackParams p) {
  __shared__ uint32_t tile[128][65];
  __shared__ int64_t qoff[kMaxMasks];
  const int64_t c0 = (int64_t)blockIdx.x * 64, t0 = (int64_t)blockIdx.y * 128;
  fill_qoff(p, qoff);
  stage_tile<T, 128>(p, t0, c0, tile);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t* out = static_cast<uint32_t*>(p.out);
  for (int cc = 0; cc < 8; ++cc) {
    const int cl = w * 8 + cc;
    const int64_t c = c0 + cl;
    if (c >= p.rows_p) break;  // warp-uniform
    XorTable tab[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const uint32_t x = tile[32 * s + lane][cl];
      uint32_t S[10];
#pragma unroll
      for (int l = 0; l < 10; ++l) S[l] = l < p.e ? __ballot_sync(0xffffffffu, (x >> l) & 1u) : 0u;
      tab[s] = build_xor_table(S, p.e, lane);
    }
    const int64_t base = (row_offset(p, c) + t0) / 32;
    for (int q0 = 0; q0 < p.P; q0 += 32) {
      const int q = q0 + lane;
      const uint32_t mk = q < p.P ? p.mask[q] : 0u;
      uint4 o;
      o.x = xor_lookup(tab[0], mk, p.e);
      o.y = xor_lookup(tab[1], mk, p.e);
      o.z = xor_lookup(tab[2], mk, p.e);
      o.w = xor_lookup(tab[3], mk, p.e);
      if (q < p.P) *reinterpret_cast<uint4*>(out + qoff[q] / 32 + base) = o;
    }
  }
}

// ---- B side, byte / nibble planes.  Tile of 32 t x 64 columns; each warp
// owns 8 columns with lane = t; e ballots give the slice words; the 2P
// (plane, 16-t half) outputs of a column are spread over the lanes.
template <typename T, bool NIB>
__global__ void __launch_bounds__(256) pack_cols_bytes(const __grid_constant__ PackParams p) {
  __shared__ uint32_t tile[32][65];
  __shared__ int64_t qoff[kMaxMasks];
  const int64_t c0 = (int64_t)blockIdx.x * 64, t0 = (int64_t)blockIdx.y * 32;
  fill_qoff(p, qoff);
  stage_tile<T, 32>(p, t0, c0, tile);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint8_t* out = static_cast<uint8_t*>(p.out);
  for (int cc = 0; cc < 8; ++cc) {
    const int cl = w * 8 + cc;
    const int64_t c = c0 + cl;
    if (c >= p.rows_p) break;  // warp-uniform
    const uint32_t x = tile[lane][cl];
    uint32_t S[10];
#pragma unroll
    for (int l = 0; l < 10; ++l) S[l] = l < p.e ? __ballot_sync(0xffffffffu, (x >> l) & 1u) : 0u;
    const XorTable tab = build_xor_table(S, p.e, lane);
    const int64_t base = row_offset(p, c) + t0;
    for (int it0 = 0; it0 < 2 * p.P; it0 += 32) {  // warp-uniform trip count (shuffles inside)
      const int it = it0 + lane;
      const int q = it >> 1, h = it & 1;
      const uint32_t mk = it < 2 * p.P ? p.mask[q] : 0u;
      const uint32_t bits = (xor_lookup(tab, mk, p.e) >> (16 * h)) & 0xFFFFu;
      if (it < 2 * p.P) {
        const int64_t o = qoff[q] + base + 16 * h;
        if (NIB) store_nibs16(out + o / 2, bits, p.one);
        else store_bytes16(out + o, bits, p.one);
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
// products selected by out_mask[s] (reduction mod f folded in).  One thread
// per (row, 32 columns): XOR the r parity words into e output slice words,
// then transpose bits into 32 elements.
template <typename T>
__global__ void __launch_bounds__(256) recombine_kernel(const __grid_constant__ RecombineParams p) {
  const int64_t nw = (p.n + 31) / 32;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = idx < p.m * nw;
  const int64_t r = live ? idx / nw : 0, w = live ? idx % nw : 0;
  uint32_t out[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (live)
    for (int q = 0; q < p.r; ++q) {
      const uint32_t pw = p.P[((int64_t)q * p.rows_p + r) * p.ldw + w];
#pragma unroll
      for (int s = 0; s < 10; ++s)
        if (s < p.e && (p.out_mask[s] >> q & 1ull)) out[s] ^= pw;
    }
  // elements c = 32 w + b, packed 4 (u8) or 2 (u16) per 32-bit word
  constexpr int PER = 4 / sizeof(T);
  constexpr int NW = 32 / PER;
  uint32_t vals[NW];
#pragma unroll
  for (int g = 0; g < NW; ++g) {
    uint32_t v = 0;
#pragma unroll
    for (int s = 0; s < 10; ++s) {
      if (s >= p.e) break;
      const uint32_t bits = (out[s] >> (PER * g)) & ((1u << PER) - 1);
      const uint32_t spread = sizeof(T) == 1 ? (bits * 0x00204081u) & 0x01010101u : (bits & 1u) | ((bits >> 1) << 16);
      v |= spread << s;
    }
    vals[g] = v;
  }
  T* C = static_cast<T*>(p.C);
  T* dst = C + r * p.ldc + 32 * w;
  const bool full = 32 * w + 32 <= p.n;
  const bool vec = full && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0);
  bool bad = false;
  if (live) {
    if (vec) {
      uint4* d4 = reinterpret_cast<uint4*>(dst);
#pragma unroll
      for (int h = 0; h < NW / 4; ++h) {
        uint4 o = make_uint4(vals[4 * h], vals[4 * h + 1], vals[4 * h + 2], vals[4 * h + 3]);
        if (p.add) {
          const uint4 old = d4[h];
          const uint32_t rep = sizeof(T) == 1 ? p.emask * 0x01010101u : p.emask * 0x00010001u;
          bad |= ((old.x | old.y | old.z | old.w) & ~rep) != 0;
          o.x ^= old.x & rep, o.y ^= old.y & rep, o.z ^= old.z & rep, o.w ^= old.w & rep;
        }
        d4[h] = o;
      }
    } else {
#pragma unroll
      for (int b = 0; b < 32; ++b) {
        if (32 * w + b < p.n) {
          uint32_t v = (vals[b / PER] >> (8 * sizeof(T) * (b % PER))) & (sizeof(T) == 1 ? 0xFFu : 0xFFFFu);
          if (p.add) {
            const uint32_t old = dst[b];
            bad |= old > p.emask;
            v ^= old & p.emask;
          }
          dst[b] = (T)v;
        }
      }
    }
  }
  flag_range(p.status, bad);
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
    const int64_t gx = p.fmt == kFmtBit ? ceil_div(p.Kp, 512 * 8) : ceil_div(p.Kp / 16, 256);
    const int64_t gy = std::min<int64_t>(p.rows_p, 65535);
    if (gx > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (gx <= 0 || gy <= 0) return cudaSuccess;
    const dim3 grid((unsigned)gx, (unsigned)gy);
    if (p.fmt == kFmtBit) {
      if (u16) pack_rows_bits<uint16_t><<<grid, 256, 0, s>>>(p);
      else pack_rows_bits<uint8_t><<<grid, 256, 0, s>>>(p);
    } else if (p.fmt == kFmtByte) {
      if (u16) pack_rows_bytes<uint16_t, false><<<grid, 256, 0, s>>>(p);
      else pack_rows_bytes<uint8_t, false><<<grid, 256, 0, s>>>(p);
    } else {
      if (u16) pack_rows_bytes<uint16_t, true><<<grid, 256, 0, s>>>(p);
      else pack_rows_bytes<uint8_t, true><<<grid, 256, 0, s>>>(p);
    }
    if (launches) ++*launches;
    return cudaGetLastError();
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
    const int64_t gy = p.Kp / 32;
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
  const int64_t n = p.m * ((p.n + 31) / 32);
  if (p.elem_bytes == 2) return launch(recombine_kernel<uint16_t>, ceil_div(n, 256), 256, s, launches, p);
  return launch(recombine_kernel<uint8_t>, ceil_div(n, 256), 256, s, launches, p);
}

}  // namespace m4rie
