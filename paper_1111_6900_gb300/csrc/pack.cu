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

__device__ __forceinline__ void flag_range(int* status, bool bad) {
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusRange);
}

// ---- Operand planes with SWAR parities.  A thread takes 16 (32 for bit
// planes) consecutive elements of one row as packed 32-bit words (4 bytes or 2
// halfwords per word) and, for every mask q, computes parity(x & mask_q) of
// all of them at once: AND with the mask replicated per element, then fold the
// element's bits onto its lowest bit (x ^= x >> 4, 2, 1 for bytes; 8, 4, 2, 1
// for halfwords; folds above the element width e are skipped).  The 0/1
// results are laid out as bytes (0 / one), nibbles or bits.  B is transposed
// first, so both sides read rows.
//
// Nibble and bit planes store the entries of each group of 8 (nibbles) or 32
// (bits) consecutive t in a fixed permuted order within the output word, the
// order that falls out of the SWAR words without shuffling bits around.  Both
// operands of a product go through this kernel, so the permutation is the
// same on both sides of every inner product and sum_t a_t b_t is unchanged.

template <typename T>
struct Swar;
template <>
struct Swar<uint8_t> {
  static constexpr int PER = 4;  // elements per word
  static __device__ __forceinline__ uint32_t rep(uint32_t m) { return m * 0x01010101u; }
  // FOLD = 1, 2, 3 folds cover elements of <= 2, 4, 8 bits
  template <int FOLD>
  static __device__ __forceinline__ uint32_t parity(uint32_t y) {
    if (FOLD >= 3) y ^= y >> 4;
    if (FOLD >= 2) y ^= y >> 2;
    y ^= y >> 1;
    return y & 0x01010101u;  // element u's parity at bit 8u
  }
};
template <>
struct Swar<uint16_t> {
  static constexpr int PER = 2;
  static __device__ __forceinline__ uint32_t rep(uint32_t m) { return m * 0x00010001u; }
  template <int FOLD>
  static __device__ __forceinline__ uint32_t parity(uint32_t y) {
    y ^= y >> 8;
    y ^= y >> 4;
    y ^= y >> 2;
    y ^= y >> 1;
    return y & 0x00010001u;  // element u's parity at bit 16u
  }
};

// Parity-fold depth for e-bit elements in T.
inline int fold_of(int e) { return e <= 2 ? 1 : e <= 4 ? 2 : 3; }

constexpr int NE = 32;  // elements per thread

// NE consecutive elements of row r from t0 (zeros past the row end), packed.
template <typename T>
__device__ __forceinline__ void load_row(const PackParams& p, int64_t r, int64_t t0, uint32_t (&v)[NE * sizeof(T) / 4]) {
  constexpr int W = NE * (int)sizeof(T) / 4;
  const T* row = static_cast<const T*>(p.X) + r * p.ldx;
  if (p.vec && t0 + NE <= p.K) {
    const uint4* q = reinterpret_cast<const uint4*>(row + t0);
#pragma unroll
    for (int k = 0; k < W / 4; ++k) {
      const uint4 a = q[k];
      v[4 * k] = a.x, v[4 * k + 1] = a.y, v[4 * k + 2] = a.z, v[4 * k + 3] = a.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < W; ++k) v[k] = 0;
#pragma unroll
    for (int u = 0; u < NE; ++u)
      if (t0 + u < p.K) v[u / Swar<T>::PER] |= (uint32_t)row[t0 + u] << (8 * sizeof(T) * (u % Swar<T>::PER));
  }
}

// Per-block tables: plane offsets qoff[q] = b*bstride + i*G*ld + j*Kp for
// q = (b*nb + i)*kb + j, and the masks replicated per packed element.
template <typename T>
__device__ __forceinline__ void plane_tables(const PackParams& p, int64_t* qoff, uint32_t* mrep) {
  for (int q = threadIdx.x; q < p.P; q += blockDim.x) {
    const int b = q / (p.nb * p.kb), i = (q / p.kb) % p.nb, j = q % p.kb;
    qoff[q] = (int64_t)b * p.bstride + (int64_t)i * (p.emajor ? 1 : p.G) * p.ld + (int64_t)j * p.Kp;
    mrep[q] = Swar<T>::rep(p.mask[q]);
  }
}

// Rows r0, r0 + rstep, ... of one plane job; this thread's elements start at
// t0 = tchunk * NE (threads with t0 >= Kp only join the warp-wide votes).
template <typename T, int FMT, int FOLD>
__device__ __forceinline__ void pack_planes_rows(const PackParams& p, const int64_t* qoff, const uint32_t* mrep,
                                                 int64_t tchunk, int64_t r0, int64_t rstep) {
  constexpr int W = NE * (int)sizeof(T) / 4;  // packed input words per thread
  const int64_t t0 = tchunk * NE;
  const bool live_t = t0 < p.Kp;
  const uint32_t erep = Swar<T>::rep(p.emask);
  for (int64_t r = r0; r < p.rows_p; r += rstep) {
    uint32_t v[W];
#pragma unroll
    for (int k = 0; k < W; ++k) v[k] = 0;
    if (live_t && r < p.rows) load_row<T>(p, r, t0, v);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      bad |= (v[k] & ~erep) != 0;
      v[k] &= erep;
    }
    flag_range(p.status, bad);
    if (!live_t) continue;
    // row offset of input row r in the plane layout (32-bit division: r < 2^31, G < 2^16)
    const uint32_t rr = (uint32_t)r, G = (uint32_t)p.G, g = rr / G;
    const int64_t base = ((int64_t)g * p.nb * G + (int64_t)(rr - g * G) * (p.emajor ? p.nb : 1)) * p.ld + t0;
    uint8_t* out = static_cast<uint8_t*>(p.out);
#pragma unroll 1
    for (int q = 0; q < p.P; ++q) {
      const uint32_t m = mrep[q];
      const int64_t o = qoff[q] + base;
      uint32_t par[W];
#pragma unroll
      for (int k = 0; k < W; ++k) par[k] = Swar<T>::template parity<FOLD>(v[k] & m);
      if (FMT == kFmtBit) {
        // parity words (element u at bit 8u or 16u) shifted by k interleave
        // into 32 distinct bits (permuted order)
        uint32_t word = 0;
#pragma unroll
        for (int k = 0; k < W; ++k) word |= par[k] << k;
        reinterpret_cast<uint32_t*>(out)[o / 32] = word;
      } else if (FMT == kFmtByte) {
        uint32_t w[8];
        if (sizeof(T) == 1) {
#pragma unroll
          for (int k = 0; k < 8; ++k) w[k] = par[k] * p.one;
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k)
            // two elements per parity word, at bits 0 and 16 -> bytes 4k .. 4k+3
            w[k] = ((par[2 * k] & 1u) | ((par[2 * k] >> 8) & 0x100u) | ((par[2 * k + 1] & 1u) << 16) |
                    ((par[2 * k + 1] >> 16) << 24)) * p.one;
        }
        uint4* d = reinterpret_cast<uint4*>(out + o);
        d[0] = make_uint4(w[0], w[1], w[2], w[3]);
        d[1] = make_uint4(w[4], w[5], w[6], w[7]);
      } else {
        // 32 entries -> 32 nibbles: parity words shifted by 4 j interleave
        // into distinct nibbles (permuted order), times `one`
        uint32_t w[4] = {0, 0, 0, 0};
        constexpr int PW = W / 4;  // parity words per output word
#pragma unroll
        for (int k = 0; k < W; ++k) w[k / PW] |= par[k] << (4 * (k % PW));
        *reinterpret_cast<uint4*>(out + o / 2) = make_uint4(w[0] * p.one, w[1] * p.one, w[2] * p.one, w[3] * p.one);
      }
    }
  }
}

// grid.x covers a row in chunks of 256 threads x NE elements, grid.y strides over rows.
template <typename T, int FMT, int FOLD>
__global__ void __launch_bounds__(256) pack_planes_kernel(const __grid_constant__ PackParams p) {
  __shared__ int64_t qoff[kMaxMasks];
  __shared__ uint32_t mrep[kMaxMasks];
  plane_tables<T>(p, qoff, mrep);
  __syncthreads();
  pack_planes_rows<T, FMT, FOLD>(p, qoff, mrep, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y,
                                 gridDim.y);
}

// Index of the job whose block range [start[j], start[j+1]) holds block b.
__device__ __forceinline__ int find_job(const int64_t* __restrict__ start, int njobs, int64_t b) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Threads per row and rows per 256-thread block of a plane job: a row of Kp
// entries needs ceil(Kp / NE) threads, rounded up to a power of two (at least
// a warp, at most the block); short rows share a block.
__host__ __device__ inline void job_shape(int64_t Kp, int ne, int64_t& tpr, int64_t& rpb, int64_t& gx) {
  const int64_t need = (Kp + ne - 1) / ne;
  tpr = 32;
  while (tpr < need && tpr < 256) tpr *= 2;
  rpb = 256 / tpr;
  gx = (need + 255) / 256;  // blocks per row when a row needs more than 256 threads
}

// Many plane jobs in one launch: block b belongs to job j with
// start[j] <= b < start[j+1]; within the job, local block l covers rows
// (l / gx) * rpb + threadIdx.x / tpr and chunk (l % gx) * 256 + threadIdx.x % tpr.
// Jobs of one launch may have different e: the fold covers the widest (8 bits
// for uint8, 16 for uint16); extra folds over zero bits change nothing.
template <typename T, int FMT>
__global__ void __launch_bounds__(256) pack_planes_batched(const PackParams* __restrict__ jobs,
                                                           const int64_t* __restrict__ start, int njobs) {
  __shared__ int64_t qoff[kMaxMasks];
  __shared__ uint32_t mrep[kMaxMasks];
  __shared__ int sj;
  if (threadIdx.x == 0) sj = find_job(start, njobs, blockIdx.x);
  __syncthreads();
  const PackParams& p = jobs[sj];
  plane_tables<T>(p, qoff, mrep);
  __syncthreads();
  int64_t tpr, rpb, gx;
  job_shape(p.Kp, NE, tpr, rpb, gx);
  const int64_t l = (int64_t)blockIdx.x - start[sj];
  const int64_t r = (l / gx) * rpb + threadIdx.x / tpr;
  const int64_t chunk = (l % gx) * 256 + threadIdx.x % tpr;
  // rows past the job's end still run the loop body's warp votes (zero data)
  pack_planes_rows<T, FMT, sizeof(T) == 1 ? 3 : 4>(p, qoff, mrep, r < p.rows_p ? chunk : (p.Kp + NE - 1) / NE,
                                                  r < p.rows_p ? r : 0, p.rows_p);
}

// ---- Element transpose X (K x rows, row-major) -> Xt (rows x K), tiles of
// 64 x 64 elements through shared memory (one 32-bit word per element).
template <typename T>
__device__ __forceinline__ void transpose_tiles(const T* __restrict__ X, int64_t ldx, int64_t K, int64_t rows,
                                                T* __restrict__ Xt, int vec, int64_t c0, int64_t ty0, int64_t tystep,
                                                uint32_t (*tile)[65]) {
  for (int64_t t0 = ty0 * 64; t0 < K; t0 += tystep * 64) {
    constexpr int CH = 64 * sizeof(T) / 16;  // 16-byte chunks per tile row
    if (vec && c0 + 64 <= rows && t0 + 64 <= K) {
      for (int idx = threadIdx.x; idx < 64 * CH; idx += 256) {
        const int tt = idx / CH, ch = idx % CH;
        const uint4 a = *reinterpret_cast<const uint4*>(X + (t0 + tt) * ldx + c0 + ch * (16 / sizeof(T)));
        const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int k = 0; k < 16 / (int)sizeof(T); ++k)
          tile[tt][ch * (16 / sizeof(T)) + k] =
              sizeof(T) == 1 ? (w[k >> 2] >> (8 * (k & 3))) & 0xFFu : (w[k >> 1] >> (16 * (k & 1))) & 0xFFFFu;
      }
    } else {
      for (int idx = threadIdx.x; idx < 64 * 64; idx += 256) {
        const int tt = idx >> 6, cc = idx & 63;
        const int64_t t = t0 + tt, c = c0 + cc;
        tile[tt][cc] = (t < K && c < rows) ? (uint32_t)X[t * ldx + c] : 0u;
      }
    }
    __syncthreads();
    // thread -> (column cl, 16 consecutive t)
    const int cl = threadIdx.x >> 2, tq = (threadIdx.x & 3) * 16;
    const int64_t c = c0 + cl;
    if (c < rows) {
      T* dst = Xt + c * K + t0 + tq;
      if (vec && t0 + tq + 16 <= K) {
        uint32_t w[16 * sizeof(T) / 4];
#pragma unroll
        for (int k = 0; k < 16 * (int)sizeof(T) / 4; ++k) {
          if (sizeof(T) == 1)
            w[k] = tile[tq + 4 * k][cl] | (tile[tq + 4 * k + 1][cl] << 8) | (tile[tq + 4 * k + 2][cl] << 16) |
                   (tile[tq + 4 * k + 3][cl] << 24);
          else
            w[k] = tile[tq + 2 * k][cl] | (tile[tq + 2 * k + 1][cl] << 16);
        }
        uint4* d4 = reinterpret_cast<uint4*>(dst);
#pragma unroll
        for (int k = 0; k < (int)sizeof(T); ++k) d4[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
      } else {
        for (int u = 0; u < 16; ++u)
          if (t0 + tq + u < K) dst[u] = (T)tile[tq + u][cl];
      }
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256) transpose_kernel(const T* __restrict__ X, int64_t ldx, int64_t K, int64_t rows,
                                                        T* __restrict__ Xt, int vec) {
  __shared__ uint32_t tile[64][65];
  transpose_tiles<T>(X, ldx, K, rows, Xt, vec, (int64_t)blockIdx.x * 64, blockIdx.y, gridDim.y, tile);
}

// Many transposes in one launch (block ranges per job as in pack_planes_batched).
template <typename T>
__global__ void __launch_bounds__(256) transpose_batched(const TransposeJob* __restrict__ jobs,
                                                         const int64_t* __restrict__ start, int njobs) {
  __shared__ uint32_t tile[64][65];
  __shared__ int sj;
  if (threadIdx.x == 0) sj = find_job(start, njobs, blockIdx.x);
  __syncthreads();
  const TransposeJob& j = jobs[sj];
  const int64_t gx = (j.rows + 63) / 64;
  const int64_t l = (int64_t)blockIdx.x - start[sj];
  transpose_tiles<T>(static_cast<const T*>(j.X), j.ldx, j.K, j.rows, static_cast<T*>(j.Xt), j.vec, (l % gx) * 64,
                     l / gx, (j.K + 63) / 64, tile);
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
// per (row, 32 columns): XOR the r parity words into E output slice words
// (which products feed which slices comes from a per-block table), then
// transpose the bits into 32 elements.
template <typename T, int E>
__global__ void __launch_bounds__(256) recombine_kernel(const __grid_constant__ RecombineParams p) {
  __shared__ uint32_t qmask[64];  // bit s: product q feeds output slice s
  for (int q = threadIdx.x; q < p.r; q += blockDim.x) {
    uint32_t m = 0;
#pragma unroll
    for (int s = 0; s < E; ++s) m |= (uint32_t)((p.out_mask[s] >> q) & 1ull) << s;
    qmask[q] = m;
  }
  __syncthreads();
  const int64_t nw = (p.n + 31) / 32;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = idx < p.m * nw;
  const int64_t r = live ? idx / nw : 0, w = live ? idx % nw : 0;
  uint32_t out[E];
#pragma unroll
  for (int s = 0; s < E; ++s) out[s] = 0;
  if (live) {
    const uint32_t* src = p.P + r * p.ldw + w;
    const int64_t pstride = p.rows_p * p.ldw;
#pragma unroll 4
    for (int q = 0; q < p.r; ++q) {
      const uint32_t pw = __ldg(src + q * pstride);
      const uint32_t m = qmask[q];
#pragma unroll
      for (int s = 0; s < E; ++s) out[s] ^= (m >> s & 1u) ? pw : 0u;
    }
  }
  // elements c = 32 w + b, packed 4 (u8) or 2 (u16) per 32-bit word
  constexpr int PER = 4 / sizeof(T);
  constexpr int NW = 32 / PER;
  uint32_t vals[NW];
#pragma unroll
  for (int g = 0; g < NW; ++g) {
    uint32_t v = 0;
#pragma unroll
    for (int s = 0; s < E; ++s) {
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

template <int FMT>
void launch_planes_fmt(const PackParams& p, dim3 grid, cudaStream_t s) {
  if (p.elem_bytes == 2) {
    pack_planes_kernel<uint16_t, FMT, 4><<<grid, 256, 0, s>>>(p);
    return;
  }
  switch (fold_of(p.e)) {
    case 1: pack_planes_kernel<uint8_t, FMT, 1><<<grid, 256, 0, s>>>(p); break;
    case 2: pack_planes_kernel<uint8_t, FMT, 2><<<grid, 256, 0, s>>>(p); break;
    default: pack_planes_kernel<uint8_t, FMT, 3><<<grid, 256, 0, s>>>(p); break;
  }
}

cudaError_t launch_pack_planes(const PackParams& p, cudaStream_t s, int64_t* launches) {
  const int64_t gx = ceil_div(ceil_div(p.Kp, NE), 256);
  const int64_t gy = std::min<int64_t>(p.rows_p, 65535);
  if (gx > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (gx <= 0 || gy <= 0) return cudaSuccess;
  const dim3 grid((unsigned)gx, (unsigned)gy);
  if (p.fmt == kFmtBit) launch_planes_fmt<kFmtBit>(p, grid, s);
  else if (p.fmt == kFmtByte) launch_planes_fmt<kFmtByte>(p, grid, s);
  else launch_planes_fmt<kFmtNib>(p, grid, s);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_transpose(const void* X, int64_t ldx, int64_t K, int64_t rows, int elem_bytes, void* Xt,
                             cudaStream_t s, int64_t* launches) {
  if (K <= 0 || rows <= 0) return cudaSuccess;
  const int64_t gx = ceil_div(rows, 64), gy = std::min<int64_t>(ceil_div(K, 64), 65535);
  if (gx > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const int vec = ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Xt)) & 15u) == 0 &&
                  (ldx * elem_bytes) % 16 == 0 && (K * elem_bytes) % 16 == 0;
  const dim3 grid((unsigned)gx, (unsigned)gy);
  if (elem_bytes == 2)
    transpose_kernel<uint16_t><<<grid, 256, 0, s>>>(static_cast<const uint16_t*>(X), ldx, K, rows,
                                                    static_cast<uint16_t*>(Xt), vec);
  else
    transpose_kernel<uint8_t><<<grid, 256, 0, s>>>(static_cast<const uint8_t*>(X), ldx, K, rows,
                                                   static_cast<uint8_t*>(Xt), vec);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_pack_batched(const PackParams* d_jobs, const int64_t* d_start, int njobs, int64_t blocks, int fmt,
                                int elem_bytes, cudaStream_t s, int64_t* launches) {
  if (njobs <= 0 || blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const unsigned g = (unsigned)blocks;
  const bool u16 = elem_bytes == 2;
  if (fmt == kFmtBit) {
    if (u16) pack_planes_batched<uint16_t, kFmtBit><<<g, 256, 0, s>>>(d_jobs, d_start, njobs);
    else pack_planes_batched<uint8_t, kFmtBit><<<g, 256, 0, s>>>(d_jobs, d_start, njobs);
  } else if (fmt == kFmtByte) {
    if (u16) pack_planes_batched<uint16_t, kFmtByte><<<g, 256, 0, s>>>(d_jobs, d_start, njobs);
    else pack_planes_batched<uint8_t, kFmtByte><<<g, 256, 0, s>>>(d_jobs, d_start, njobs);
  } else {
    if (u16) pack_planes_batched<uint16_t, kFmtNib><<<g, 256, 0, s>>>(d_jobs, d_start, njobs);
    else pack_planes_batched<uint8_t, kFmtNib><<<g, 256, 0, s>>>(d_jobs, d_start, njobs);
  }
  if (launches) ++*launches;
  return cudaGetLastError();
}

int64_t pack_job_blocks(const PackParams& p) {
  int64_t tpr, rpb, gx;
  job_shape(p.Kp, NE, tpr, rpb, gx);
  return gx * ceil_div(p.rows_p, rpb);
}

int64_t transpose_job_blocks(const TransposeJob& j) { return ceil_div(j.rows, 64) * ceil_div(j.K, 64); }

cudaError_t launch_transpose_batched(const TransposeJob* d_jobs, const int64_t* d_start, int njobs, int64_t blocks,
                                     int elem_bytes, cudaStream_t s, int64_t* launches) {
  if (njobs <= 0 || blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (elem_bytes == 2) transpose_batched<uint16_t><<<(unsigned)blocks, 256, 0, s>>>(d_jobs, d_start, njobs);
  else transpose_batched<uint8_t><<<(unsigned)blocks, 256, 0, s>>>(d_jobs, d_start, njobs);
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
  const int64_t g = ceil_div(n, 256);
  if (p.r > 64) return cudaErrorInvalidValue;
  switch (p.e) {
    case 2: return launch(recombine_kernel<uint8_t, 2>, g, 256, s, launches, p);
    case 3: return launch(recombine_kernel<uint8_t, 3>, g, 256, s, launches, p);
    case 4: return launch(recombine_kernel<uint8_t, 4>, g, 256, s, launches, p);
    case 5: return launch(recombine_kernel<uint8_t, 5>, g, 256, s, launches, p);
    case 6: return launch(recombine_kernel<uint8_t, 6>, g, 256, s, launches, p);
    case 7: return launch(recombine_kernel<uint8_t, 7>, g, 256, s, launches, p);
    case 8: return launch(recombine_kernel<uint8_t, 8>, g, 256, s, launches, p);
    case 9: return launch(recombine_kernel<uint16_t, 9>, g, 256, s, launches, p);
    case 10: return launch(recombine_kernel<uint16_t, 10>, g, 256, s, launches, p);
  }
  return cudaErrorInvalidValue;
}

}  // namespace m4rie
