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

// ---- Operand planes from bit slices.  Every plane entry parity(x & mask) is
// a GF(2)-linear function of the bits of x: it is the XOR, over the bits i set
// in the mask, of bit i of x.  A thread takes NE = 32 consecutive elements of
// one row as packed 32-bit words (4 bytes or 2 halfwords per word), turns
// them into bit slices (slice i = bit i of all 32 elements, one word) with a
// SWAR bit-matrix transpose, and then forms each plane word as the XOR of the
// slices its mask selects (one LOP3 per bit).  The 0/1 results are laid out as
// bits, bytes (0 / one) or nibbles (0 / one).  A side's plane rows may be the
// rows of X (pack_planes_rows) or its columns (pack_planes_cols).
//
// The 32 entries of a plane word come out in a fixed permuted order of t
// (slice bit 8u + k, or 16u + k for halfwords, is element u of packed word
// k), and the byte and nibble layouts spread the bits in their own fixed
// order.  Both operands of a product go through these kernels, so the
// permutation is the same on both sides of every inner product and
// sum_t a_t b_t is unchanged.

template <typename T>
struct Swar;
template <>
struct Swar<uint8_t> {
  static constexpr int PER = 4;  // elements per word
  static __device__ __forceinline__ uint32_t rep(uint32_t m) { return m * 0x01010101u; }
};
template <>
struct Swar<uint16_t> {
  static constexpr int PER = 2;
  static __device__ __forceinline__ uint32_t rep(uint32_t m) { return m * 0x00010001u; }
};

constexpr int NE = 32;  // elements per thread

// Exchange bit i + D of a with bit i of b for the bit positions i in M (the
// lower half of every 2D-bit block): one step of the recursive transpose.
template <int D, uint32_t M>
__device__ __forceinline__ void delta_swap(uint32_t& a, uint32_t& b) {
  const uint32_t t = ((a >> D) ^ b) & M;
  b ^= t;
  a ^= t << D;
}
// The same step when bits i + D of a and all bits of b outside M are known to
// be zero: only a receives data (b is not needed afterwards).
template <int D>
__device__ __forceinline__ void delta_merge(uint32_t& a, uint32_t b) {
  a |= b << D;
}

// In place: v[k] holds elements PER k .. PER k + PER - 1 of E bits; afterwards
// v[i] (i < E) is bit slice i, its bit 8u + k (bytes) or 16u + k (halfwords)
// taken from element u of the input word k.  This transposes the (word k,
// bit i) bit matrix of every element lane at once.  Bits at and above E are
// zero on input, so for E <= 4 (E <= 2) the first one (two) steps only merge
// words and the upper words are dropped.
template <typename T, int E>
__device__ __forceinline__ void bit_slices(uint32_t (&v)[NE * sizeof(T) / 4]) {
  if constexpr (sizeof(T) == 1) {
    if constexpr (E > 4) {
#pragma unroll
      for (int k = 0; k < 4; ++k) delta_swap<4, 0x0F0F0F0Fu>(v[k], v[k + 4]);
#pragma unroll
      for (int k : {0, 1, 4, 5}) delta_swap<2, 0x33333333u>(v[k], v[k + 2]);
#pragma unroll
      for (int k : {0, 2, 4, 6}) delta_swap<1, 0x55555555u>(v[k], v[k + 1]);
    } else if constexpr (E > 2) {
#pragma unroll
      for (int k = 0; k < 4; ++k) delta_merge<4>(v[k], v[k + 4]);
      delta_swap<2, 0x33333333u>(v[0], v[2]);
      delta_swap<2, 0x33333333u>(v[1], v[3]);
      delta_swap<1, 0x55555555u>(v[0], v[1]);
      delta_swap<1, 0x55555555u>(v[2], v[3]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) delta_merge<4>(v[k], v[k + 4]);
      delta_merge<2>(v[0], v[2]);
      delta_merge<2>(v[1], v[3]);
      delta_swap<1, 0x55555555u>(v[0], v[1]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) delta_swap<8, 0x00FF00FFu>(v[k], v[k + 8]);
#pragma unroll
    for (int k : {0, 1, 2, 3, 8, 9, 10, 11}) delta_swap<4, 0x0F0F0F0Fu>(v[k], v[k + 4]);
#pragma unroll
    for (int k : {0, 1, 4, 5, 8, 9, 12, 13}) delta_swap<2, 0x33333333u>(v[k], v[k + 2]);
#pragma unroll
    for (int k : {0, 2, 4, 6, 8, 10, 12, 14}) delta_swap<1, 0x55555555u>(v[k], v[k + 1]);
  }
}

// Mask words per plane in the shared table: bit i of the mask as 0 / ~0,
// padded to whole 128-bit loads.
template <int E>
__host__ __device__ constexpr int mask_words() { return (E + 3) & ~3; }

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

// Per-block table: the masks expanded to one 0 / ~0 word per bit.
template <int E>
__device__ __forceinline__ void plane_tables(const PackParams& p, uint32_t* mexp) {
  constexpr int MW = mask_words<E>();
  for (int x = threadIdx.x; x < p.P * MW; x += blockDim.x) {
    const int q = x / MW, i = x % MW;
    mexp[x] = (i < E && ((p.mask[q] >> i) & 1u)) ? ~0u : 0u;
  }
}

// All planes of NE consecutive entries (from t0) of input row r, given its
// packed elements v (bits at and above E zero); v is turned into bit slices.
template <typename T, int FMT, int E>
__device__ __forceinline__ void plane_out(const PackParams& p, const uint32_t* mexp, int64_t r, int64_t t0,
                                          uint32_t (&v)[NE * sizeof(T) / 4]) {
  constexpr int MW = mask_words<E>();
  constexpr int BITS = FMT == kFmtBit ? 1 : FMT == kFmtByte ? 8 : 4;  // per entry
  bit_slices<T, E>(v);
  // entry offset of input row r, entry t0 in the plane layout (r < 2^31, G < 512)
  const uint32_t rr = (uint32_t)r, G = (uint32_t)p.G, g = (uint32_t)(((uint64_t)rr * p.gmul) >> 40);
  const uint64_t base =
      ((uint64_t)g * p.nb * G + (uint64_t)(rr - g * G) * (p.emajor ? p.nb : 1)) * p.ld + (uint64_t)t0;
  uint8_t* const rowp = static_cast<uint8_t*>(p.out) + base * BITS / 8;
#pragma unroll 1
  for (int q = 0; q < p.P; ++q) {
    const uint4* mq = reinterpret_cast<const uint4*>(mexp + q * MW);
    uint32_t x = 0;
#pragma unroll
    for (int i4 = 0; i4 < MW; i4 += 4) {
      const uint4 mb = mq[i4 / 4];
      const uint32_t mw[4] = {mb.x, mb.y, mb.z, mb.w};
#pragma unroll
      for (int i = i4; i < i4 + 4 && i < E; ++i) x ^= v[i] & mw[i - i4];
    }
    uint8_t* const dst = rowp + p.qoff[q];
    if (FMT == kFmtBit) {
      *reinterpret_cast<uint32_t*>(dst) = x;
    } else if (FMT == kFmtByte) {
      // byte j of word k <- bit 8j + k
      uint32_t w[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) w[k] = ((x >> k) & 0x01010101u) * p.one;
      uint4* d = reinterpret_cast<uint4*>(dst);
      d[0] = make_uint4(w[0], w[1], w[2], w[3]);
      d[1] = make_uint4(w[4], w[5], w[6], w[7]);
    } else {
      // nibble j of word k <- bit 4j + k
      uint32_t w[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) w[k] = ((x >> k) & 0x11111111u) * p.one;
      *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// Rows r0, r0 + rstep, ... of one plane job; this thread's elements start at
// t0 = tchunk * NE (threads with t0 >= Kp only join the warp-wide votes).
template <typename T, int FMT, int E>
__device__ __forceinline__ void pack_planes_rows(const PackParams& p, const uint32_t* mexp, int64_t tchunk, int64_t r0,
                                                 int64_t rstep) {
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
    plane_out<T, FMT, E>(p, mexp, r, t0, v);
  }
}

// Shared mask table of a plane kernel (room for the largest E, 10).
struct PlaneSmem {
  uint32_t mexp[kMaxMasks * 12];
};

// A block holds 256 / tpr rows of tpr threads (tpr a power of two in
// [32, 256], at least ceil(Kp / NE) when a row fits in one block); grid.x
// covers longer rows in chunks of 256 threads x NE elements, grid.y strides
// over row groups.
template <typename T, int FMT, int E>
__device__ __forceinline__ void rows_body(const PackParams& p, int tpr, uint32_t bx, uint32_t by, uint32_t gy,
                                          uint32_t* mexp) {
  plane_tables<E>(p, mexp);
  __syncthreads();
  const int rpb = 256 / tpr;
  pack_planes_rows<T, FMT, E>(p, mexp, (int64_t)bx * 256 + threadIdx.x % tpr, (int64_t)by * rpb + threadIdx.x / tpr,
                              (int64_t)gy * rpb);
}

template <typename T, int FMT, int E>
__global__ void __launch_bounds__(256) pack_planes_kernel(const __grid_constant__ PackParams p, int tpr) {
  __shared__ PlaneSmem sm;
  pdl_enter();
  rows_body<T, FMT, E>(p, tpr, blockIdx.x, blockIdx.y, gridDim.y, sm.mexp);
}

// ---- Operand planes of the columns of X (X is K x rows, row-major; plane
// row c holds column c, so B needs no separate transpose).  A tile of 128 t x
// 64 columns passes through shared memory: each thread loads 8 bytes from each
// of 4 (u8) or 2 (u16) consecutive rows and turns them, by byte (halfword)
// permutes, into words that hold consecutive t of one column, stored column by
// column.  Then each thread takes 32 consecutive t of one column and builds
// their planes exactly as pack_planes_rows does for a row.
template <typename T>
__device__ __forceinline__ void transpose_words(const uint32_t (&r)[4 / sizeof(T)], uint32_t (&o)[4 / sizeof(T)]) {
  if constexpr (sizeof(T) == 1) {
    // 4 x 4 bytes: byte i of o[j] = byte j of r[i]
    const uint32_t a = __byte_perm(r[0], r[1], 0x5140), b = __byte_perm(r[2], r[3], 0x5140);
    const uint32_t c = __byte_perm(r[0], r[1], 0x7362), d = __byte_perm(r[2], r[3], 0x7362);
    o[0] = __byte_perm(a, b, 0x5410);
    o[1] = __byte_perm(a, b, 0x7632);
    o[2] = __byte_perm(c, d, 0x5410);
    o[3] = __byte_perm(c, d, 0x7632);
  } else {
    // 2 x 2 halfwords: halfword i of o[j] = halfword j of r[i]
    o[0] = __byte_perm(r[0], r[1], 0x5410);
    o[1] = __byte_perm(r[0], r[1], 0x7632);
  }
}

// Shared words of the column kernel's tile.
template <typename T>
__host__ __device__ constexpr int col_tile_words() { return 64 * (128 / (4 / (int)sizeof(T)) + 1); }

// Block (bx, by) of a grid with gy rows of blocks: column tile bx, t tiles
// by, by + gy, ...
template <typename T, int FMT, int E>
__device__ __forceinline__ void cols_body(const PackParams& p, uint32_t bx, uint32_t by, uint32_t gy, uint32_t* mexp,
                                          uint32_t* tile) {
  constexpr int PER = 4 / sizeof(T);       // elements per word
  constexpr int TT = 128, TC = 64;         // tile: t x columns
  constexpr int WPC = TT / PER;            // words per tile column
  constexpr int PITCH = WPC + 1;           // odd pitch: conflict-free column stores and reads
  constexpr int CPT = 8 / sizeof(T);       // columns per load task (8 bytes of a row)
  constexpr int CG = TC / CPT;             // column groups: 8 (u8), 16 (u16)
  constexpr int PASSES = WPC * CG / 256;   // 1 (u8), 4 (u16)
  constexpr int W = NE * (int)sizeof(T) / 4;
  static_assert(TC * PITCH == col_tile_words<T>(), "tile size");
  plane_tables<E>(p, mexp);
  const T* X = static_cast<const T*>(p.X);
  const int64_t c0 = (int64_t)bx * TC;
  const bool aligned8 = ((reinterpret_cast<uintptr_t>(X) | (uintptr_t)(p.ldx * sizeof(T))) & 7u) == 0;
  const uint32_t erep = Swar<T>::rep(p.emask);
  for (int64_t tt0 = (int64_t)by * TT; tt0 < p.Kp; tt0 += (int64_t)gy * TT) {
    const bool fast = aligned8 && c0 + TC <= p.rows && tt0 + TT <= p.K;
#pragma unroll
    for (int pass = 0; pass < PASSES; ++pass) {
      // a warp takes 8 column groups x 4 row groups
      const int cg = (threadIdx.x & 7) + 8 * (pass % (CG / 8));
      const int rg = (threadIdx.x >> 3) + 32 * (pass / (CG / 8));
      uint32_t lo[PER], hi[PER];
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        const int64_t t = tt0 + (int64_t)rg * PER + i, c = c0 + (int64_t)cg * CPT;
        if (fast) {
          const uint2 a = *reinterpret_cast<const uint2*>(X + t * p.ldx + c);
          lo[i] = a.x, hi[i] = a.y;
        } else {
          lo[i] = hi[i] = 0;
          if (t < p.K) {
#pragma unroll
            for (int u = 0; u < CPT; ++u)
              if (c + u < p.rows) {
                const uint32_t x = (uint32_t)X[t * p.ldx + c + u] << (8 * sizeof(T) * (u % PER));
                if (u < PER) lo[i] |= x;
                else hi[i] |= x;
              }
          }
        }
      }
      uint32_t o[PER];
      transpose_words<T>(lo, o);
#pragma unroll
      for (int j = 0; j < PER; ++j) tile[(cg * CPT + j) * PITCH + rg] = o[j];
      transpose_words<T>(hi, o);
#pragma unroll
      for (int j = 0; j < PER; ++j) tile[(cg * CPT + PER + j) * PITCH + rg] = o[j];
    }
    __syncthreads();
    // thread -> (column cl, 32 consecutive t from t0)
    const int cl = threadIdx.x >> 2, ch = threadIdx.x & 3;
    uint32_t v[W];
#pragma unroll
    for (int k = 0; k < W; ++k) v[k] = tile[cl * PITCH + ch * W + k];
    __syncthreads();
    bool bad = false;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      bad |= (v[k] & ~erep) != 0;
      v[k] &= erep;
    }
    flag_range(p.status, bad);
    const int64_t r = c0 + cl, t0 = tt0 + (int64_t)ch * NE;
    if (r < p.rows_p && t0 < p.Kp) plane_out<T, FMT, E>(p, mexp, r, t0, v);
  }
}

template <typename T, int FMT, int E>
__global__ void __launch_bounds__(256) pack_planes_cols(const __grid_constant__ PackParams p) {
  __shared__ PlaneSmem sm;
  __shared__ uint32_t tile[col_tile_words<T>()];
  pdl_enter();
  cols_body<T, FMT, E>(p, blockIdx.x, blockIdx.y, gridDim.y, sm.mexp, tile);
}

// Both operands of a product in one launch: blocks [0, gxa * gya) run the row
// kernel on pa (A), the others the column kernel on pb (B), so the two sides
// stream concurrently.
template <typename T, int FMT, int E>
__global__ void __launch_bounds__(256) pack_planes_pair(const __grid_constant__ PackParams pa, int tpr, uint32_t gxa,
                                                        uint32_t gya, const __grid_constant__ PackParams pb,
                                                        uint32_t gxb, uint32_t gyb) {
  __shared__ PlaneSmem sm;
  __shared__ uint32_t tile[col_tile_words<T>()];
  pdl_enter();
  const uint32_t b = blockIdx.x, na = gxa * gya;
  if (b < na) {
    rows_body<T, FMT, E>(pa, tpr, b % gxa, b / gxa, gya, sm.mexp);
  } else {
    const uint32_t bb = b - na;
    cols_body<T, FMT, E>(pb, bb % gxb, bb / gxb, gyb, sm.mexp, tile);
  }
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
// Jobs of one launch may have different e: the bit slices cover the widest (8
// bits for uint8, 10 for uint16); slices of bits above a job's e are zero and
// its masks never select them.
template <typename T, int FMT>
__global__ void __launch_bounds__(256) pack_planes_batched(const PackParams* __restrict__ jobs,
                                                           const int64_t* __restrict__ start, int njobs) {
  constexpr int E = sizeof(T) == 1 ? 8 : 10;
  __shared__ PlaneSmem sm;
  __shared__ int sj;
  if (threadIdx.x == 0) sj = find_job(start, njobs, blockIdx.x);
  __syncthreads();
  const PackParams& p = jobs[sj];
  plane_tables<E>(p, sm.mexp);
  __syncthreads();
  int64_t tpr, rpb, gx;
  job_shape(p.Kp, NE, tpr, rpb, gx);
  const int64_t l = (int64_t)blockIdx.x - start[sj];
  const int64_t r = (l / gx) * rpb + threadIdx.x / tpr;
  const int64_t chunk = (l % gx) * 256 + threadIdx.x % tpr;
  // rows past the job's end still run the loop body's warp votes (zero data)
  pack_planes_rows<T, FMT, E>(p, sm.mexp, r < p.rows_p ? chunk : (p.Kp + NE - 1) / NE,
                              r < p.rows_p ? r : 0, p.rows_p);
}

// Column planes of many jobs in one launch (the B operands of a batch, read
// by columns through shared memory, no transpose): block b belongs to job j
// with start[j] <= b < start[j+1] and covers its column tile l % gx, k tiles
// l / gx, l / gx + gy, ... (l = b - start[j], gx, gy as in launch_pack_cols).
__host__ __device__ inline void cols_shape(const PackParams& p, int64_t& gx, int64_t& gy) {
  gx = (p.rows_p + 63) / 64;
  gy = (p.Kp + 127) / 128;
  if (gy > 65535) gy = 65535;
}

template <typename T, int FMT>
__global__ void __launch_bounds__(256) pack_cols_batched(const PackParams* __restrict__ jobs,
                                                         const int64_t* __restrict__ start, int njobs) {
  constexpr int E = sizeof(T) == 1 ? 8 : 10;
  __shared__ PlaneSmem sm;
  __shared__ uint32_t tile[col_tile_words<T>()];
  __shared__ int sj;
  if (threadIdx.x == 0) sj = find_job(start, njobs, blockIdx.x);
  __syncthreads();
  const PackParams& p = jobs[sj];
  int64_t gx, gy;
  cols_shape(p, gx, gy);
  const int64_t l = (int64_t)blockIdx.x - start[sj];
  cols_body<T, FMT, E>(p, (uint32_t)(l % gx), (uint32_t)(l / gx), (uint32_t)gy, sm.mexp, tile);
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
// per (row, 4 words of 32 columns): it loads the r parity planes' 4 words with
// 16-byte loads (row layout: rows padded to whole 16-byte groups; blocked
// layout: half of a block row of 8 words), XORs them
// into E output slice words each (which products feed which slices comes from
// a per-block table), then transposes the bits into elements.
template <typename T, int E>
__device__ __forceinline__ bool store_elements(const RecombineParams& p, int64_t r, int64_t cs, int nc,
                                               const uint32_t* out) {
  // elements c = cs + b for b < nc <= 32, packed 4 (u8) or 2 (u16) per 32-bit word
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
  T* dst = C + r * p.ldc + cs;
  // 16-byte chunks of EPC elements: a whole chunk inside the word and the
  // matrix goes out as one vector store, a ragged one element by element
  constexpr int EPC = 16 / sizeof(T);
  const bool al = (reinterpret_cast<uintptr_t>(dst) & 15u) == 0;
  const uint32_t rep = sizeof(T) == 1 ? p.emask * 0x01010101u : p.emask * 0x00010001u;
  bool bad = false;
#pragma unroll
  for (int h = 0; h < NW / 4; ++h) {
    const int b0 = h * EPC;
    if (al && b0 + EPC <= nc && cs + b0 + EPC <= p.n) {
      uint4* d4 = reinterpret_cast<uint4*>(dst + b0);
      uint4 o = make_uint4(vals[4 * h], vals[4 * h + 1], vals[4 * h + 2], vals[4 * h + 3]);
      if (p.add) {
        const uint4 old = *d4;
        bad |= ((old.x | old.y | old.z | old.w) & ~rep) != 0;
        o.x ^= old.x & rep, o.y ^= old.y & rep, o.z ^= old.z & rep, o.w ^= old.w & rep;
      }
      *d4 = o;
    } else {
#pragma unroll
      for (int b = b0; b < b0 + EPC; ++b) {
        if (b < nc && cs + b < p.n) {
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
  return bad;
}

// Recombination of the r parity planes of one product into its elements;
// idx: this thread's index within the product, qmask: bit s of qmask[q] says
// that product q feeds output slice s.
template <typename T, int E>
__device__ __forceinline__ void recombine_body(const RecombineParams& p, int64_t idx, const uint32_t* qmask) {
  // blocked layout: 256 consecutive threads take one block (128 rows of one
  // column tile), thread 2 i + h row i's half h, so that their loads are
  // contiguous; row layout: consecutive threads along a row
  const int64_t nw = (p.n + 31) / 32, ng = p.blocked ? 2 * p.tiles_n : (nw + 3) / 4;
  int64_t r, g;
  bool live;
  if (p.blocked) {
    const int64_t blk = idx >> 8;
    r = (blk / p.tiles_n) * 128 + ((idx & 255) >> 1);
    g = 2 * (blk % p.tiles_n) + (idx & 1);
    live = r < p.m;
  } else {
    live = idx < p.m * ng;
    r = live ? idx / ng : 0;
    g = live ? idx % ng : 0;
  }
  if (!live) r = g = 0;
  // output column of word u = 0, and this thread's columns within its tile
  const int64_t cs0 = p.blocked ? (g >> 1) * p.tcols + 128 * (g & 1) : 128 * g;
  const int tc = p.blocked ? p.tcols - 128 * (int)(g & 1) : 128;
  uint32_t out[4][E];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int s = 0; s < E; ++s) out[u][s] = 0;
  if (live) {
    const uint32_t* base = p.blocked ? p.P + ((r >> 7) * p.tiles_n + (g >> 1)) * 1024 + (r & 127) * 8 + 4 * (g & 1)
                                     : p.P + r * p.ldw + 4 * g;
    const uint4* src = reinterpret_cast<const uint4*>(base);
    const int64_t pstride = (p.blocked ? p.bstride : p.rows_p * p.ldw) / 4;  // in 16-byte groups
#pragma unroll 8
    for (int q = 0; q < p.r; ++q) {
      const uint4 pw = __ldg(src + q * pstride);
      const uint32_t m = qmask[q];
#pragma unroll
      for (int s = 0; s < E; ++s)
        if ((m >> s) & 1u) {
          out[0][s] ^= pw.x;
          out[1][s] ^= pw.y;
          out[2][s] ^= pw.z;
          out[3][s] ^= pw.w;
        }
    }
  }
  bool bad = false;
  if (live) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int nc = min(32, tc - 32 * u);
      if (nc > 0 && cs0 + 32 * u < p.n) bad |= store_elements<T, E>(p, r, cs0 + 32 * u, nc, out[u]);
    }
  }
  flag_range(p.status, bad);
}

template <typename T, int E>
__global__ void __launch_bounds__(256) recombine_kernel(const __grid_constant__ RecombineParams p) {
  __shared__ uint32_t qmask[64];  // bit s: product q feeds output slice s
  pdl_enter();
  for (int q = threadIdx.x; q < p.r; q += blockDim.x) {
    uint32_t m = 0;
#pragma unroll
    for (int s = 0; s < E; ++s) m |= (uint32_t)((p.out_mask[s] >> q) & 1ull) << s;
    qmask[q] = m;
  }
  __syncthreads();
  recombine_body<T, E>(p, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, qmask);
}

// Many products' recombinations in one launch (the batched Karatsuba
// products): block b serves job find_job(start, b).
template <typename T>
__global__ void __launch_bounds__(256) recombine_batched(const RecombineParams* __restrict__ jobs,
                                                         const int64_t* __restrict__ start, int njobs) {
  constexpr int E = sizeof(T) == 1 ? 8 : 10;
  __shared__ uint32_t qmask[64];
  __shared__ int sj;
  if (threadIdx.x == 0) sj = find_job(start, njobs, blockIdx.x);
  __syncthreads();
  const RecombineParams& p = jobs[sj];
  for (int q = threadIdx.x; q < p.r; q += blockDim.x) {
    uint32_t m = 0;
#pragma unroll
    for (int s = 0; s < E; ++s) m |= (uint32_t)((p.out_mask[s] >> q) & 1ull) << s;
    qmask[q] = m;
  }
  __syncthreads();
  recombine_body<T, E>(p, ((int64_t)blockIdx.x - start[sj]) * blockDim.x + threadIdx.x, qmask);
}

template <typename K, typename... Args>
cudaError_t launch(K kernel, int64_t blocks, int threads, cudaStream_t s, int64_t* launches, Args... args) {
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  kernel<<<(unsigned)blocks, threads, 0, s>>>(args...);
  if (launches) ++*launches;
  return cudaGetLastError();
}

template <typename... Params, typename... Args>
cudaError_t launch_pdl(void (*kernel)(Params...), int64_t blocks, int threads, cudaStream_t s, int64_t* launches,
                       bool pdl, Args... args) {
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  cudaError_t err = launch_ex(kernel, dim3((unsigned)blocks), dim3(threads), 0, s, pdl, args...);
  if (launches) ++*launches;
  return err != cudaSuccess ? err : cudaGetLastError();
}

}  // namespace

// Slice counts the plane kernels are built for: e = 2, 3..4, 5..8 (bytes),
// 9..10 (halfwords).  A kernel built for more slices than e computes zero
// slices that no mask selects.
template <int FMT>
void launch_planes_fmt(const PackParams& p, dim3 grid, int tpr, cudaStream_t s) {
  const bool pdl = p.pdl != 0;
  if (p.elem_bytes == 2) launch_ex(pack_planes_kernel<uint16_t, FMT, 10>, grid, 256, 0, s, pdl, p, tpr);
  else if (p.e <= 2) launch_ex(pack_planes_kernel<uint8_t, FMT, 2>, grid, 256, 0, s, pdl, p, tpr);
  else if (p.e <= 4) launch_ex(pack_planes_kernel<uint8_t, FMT, 4>, grid, 256, 0, s, pdl, p, tpr);
  else launch_ex(pack_planes_kernel<uint8_t, FMT, 8>, grid, 256, 0, s, pdl, p, tpr);
}

bool plane_offsets(PackParams& p) {
  if (p.G < 1 || p.G >= 512 || p.P < 0 || p.P > kMaxMasks) return false;
  const int bits = p.fmt == kFmtBit ? 1 : p.fmt == kFmtByte ? 8 : 4;
  for (int q = 0; q < p.P; ++q) {
    const int b = q / (p.nb * p.kb), i = (q / p.kb) % p.nb, j = q % p.kb;
    const int64_t entries = (int64_t)b * p.bstride + (int64_t)i * (p.emajor ? 1 : p.G) * p.ld + (int64_t)j * p.Kp;
    p.qoff[q] = entries * bits / 8;
  }
  p.gmul = ((1ull << 40) + (uint64_t)p.G - 1) / (uint64_t)p.G;
  return true;
}

cudaError_t launch_pack_planes(const PackParams& p0, cudaStream_t s, int64_t* launches) {
  PackParams p = p0;
  if (!plane_offsets(p)) return cudaErrorInvalidValue;
  int64_t tpr, rpb, gx;
  job_shape(p.Kp, NE, tpr, rpb, gx);
  const int64_t gy = std::min<int64_t>(ceil_div(p.rows_p, rpb), 65535);
  if (gx > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (gx <= 0 || gy <= 0) return cudaSuccess;
  const dim3 grid((unsigned)gx, (unsigned)gy);
  if (p.fmt == kFmtBit) launch_planes_fmt<kFmtBit>(p, grid, (int)tpr, s);
  else if (p.fmt == kFmtByte) launch_planes_fmt<kFmtByte>(p, grid, (int)tpr, s);
  else launch_planes_fmt<kFmtNib>(p, grid, (int)tpr, s);
  if (launches) ++*launches;
  return cudaGetLastError();
}

template <int FMT>
void launch_cols_fmt(const PackParams& p, dim3 grid, cudaStream_t s) {
  const bool pdl = p.pdl != 0;
  if (p.elem_bytes == 2) launch_ex(pack_planes_cols<uint16_t, FMT, 10>, grid, 256, 0, s, pdl, p);
  else if (p.e <= 2) launch_ex(pack_planes_cols<uint8_t, FMT, 2>, grid, 256, 0, s, pdl, p);
  else if (p.e <= 4) launch_ex(pack_planes_cols<uint8_t, FMT, 4>, grid, 256, 0, s, pdl, p);
  else launch_ex(pack_planes_cols<uint8_t, FMT, 8>, grid, 256, 0, s, pdl, p);
}

cudaError_t launch_pack_cols(const PackParams& p0, cudaStream_t s, int64_t* launches) {
  PackParams p = p0;
  if (!plane_offsets(p)) return cudaErrorInvalidValue;
  const int64_t gx = ceil_div(p.rows_p, 64), gy = std::min<int64_t>(ceil_div(p.Kp, 128), 65535);
  if (gx > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (gx <= 0 || gy <= 0) return cudaSuccess;
  const dim3 grid((unsigned)gx, (unsigned)gy);
  if (p.fmt == kFmtBit) launch_cols_fmt<kFmtBit>(p, grid, s);
  else if (p.fmt == kFmtByte) launch_cols_fmt<kFmtByte>(p, grid, s);
  else launch_cols_fmt<kFmtNib>(p, grid, s);
  if (launches) ++*launches;
  return cudaGetLastError();
}

template <int FMT>
void launch_pair_fmt(const PackParams& a, int tpr, uint32_t gxa, uint32_t gya, const PackParams& b, uint32_t gxb,
                     uint32_t gyb, unsigned grid, cudaStream_t s) {
  const bool pdl = a.pdl != 0;
  const dim3 g(grid);
  if (a.elem_bytes == 2) launch_ex(pack_planes_pair<uint16_t, FMT, 10>, g, 256, 0, s, pdl, a, tpr, gxa, gya, b, gxb, gyb);
  else if (a.e <= 2) launch_ex(pack_planes_pair<uint8_t, FMT, 2>, g, 256, 0, s, pdl, a, tpr, gxa, gya, b, gxb, gyb);
  else if (a.e <= 4) launch_ex(pack_planes_pair<uint8_t, FMT, 4>, g, 256, 0, s, pdl, a, tpr, gxa, gya, b, gxb, gyb);
  else launch_ex(pack_planes_pair<uint8_t, FMT, 8>, g, 256, 0, s, pdl, a, tpr, gxa, gya, b, gxb, gyb);
}

cudaError_t launch_pack_pair(const PackParams& a0, const PackParams& b0, cudaStream_t s, int64_t* launches) {
  if (a0.fmt != b0.fmt || a0.e != b0.e || a0.elem_bytes != b0.elem_bytes) {
    cudaError_t err = launch_pack_planes(a0, s, launches);
    return err != cudaSuccess ? err : launch_pack_cols(b0, s, launches);
  }
  PackParams a = a0, b = b0;
  if (!plane_offsets(a) || !plane_offsets(b)) return cudaErrorInvalidValue;
  int64_t tpr, rpb, gxa;
  job_shape(a.Kp, NE, tpr, rpb, gxa);
  const int64_t gya = std::min<int64_t>(ceil_div(a.rows_p, rpb), 65535);
  const int64_t gxb = ceil_div(b.rows_p, 64), gyb = std::min<int64_t>(ceil_div(b.Kp, 128), 65535);
  const int64_t na = gxa * gya, nb = gxb * gyb;
  if (na <= 0 || nb <= 0) {  // one side empty: the single launchers handle it
    cudaError_t err = launch_pack_planes(a0, s, launches);
    return err != cudaSuccess ? err : launch_pack_cols(b0, s, launches);
  }
  if (na + nb > 0x7fffffffLL || gxa > 0xffffffffLL) return cudaErrorInvalidConfiguration;
  const unsigned grid = (unsigned)(na + nb);
  if (a.fmt == kFmtBit) launch_pair_fmt<kFmtBit>(a, (int)tpr, (uint32_t)gxa, (uint32_t)gya, b, (uint32_t)gxb, (uint32_t)gyb, grid, s);
  else if (a.fmt == kFmtByte)
    launch_pair_fmt<kFmtByte>(a, (int)tpr, (uint32_t)gxa, (uint32_t)gya, b, (uint32_t)gxb, (uint32_t)gyb, grid, s);
  else launch_pair_fmt<kFmtNib>(a, (int)tpr, (uint32_t)gxa, (uint32_t)gya, b, (uint32_t)gxb, (uint32_t)gyb, grid, s);
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

int64_t cols_job_blocks(const PackParams& p) {
  int64_t gx, gy;
  cols_shape(p, gx, gy);
  return gx * gy;
}

cudaError_t launch_cols_batched(const PackParams* d_jobs, const int64_t* d_start, int njobs, int64_t blocks, int fmt,
                                int elem_bytes, cudaStream_t s, int64_t* launches) {
  if (njobs <= 0 || blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const unsigned g = (unsigned)blocks;
  const bool u16 = elem_bytes == 2;
  if (fmt == kFmtBit) {
    if (u16) pack_cols_batched<uint16_t, kFmtBit><<<g, 256, 0, s>>>(d_jobs, d_start, njobs);
    else pack_cols_batched<uint8_t, kFmtBit><<<g, 256, 0, s>>>(d_jobs, d_start, njobs);
  } else if (fmt == kFmtByte) {
    if (u16) pack_cols_batched<uint16_t, kFmtByte><<<g, 256, 0, s>>>(d_jobs, d_start, njobs);
    else pack_cols_batched<uint8_t, kFmtByte><<<g, 256, 0, s>>>(d_jobs, d_start, njobs);
  } else {
    if (u16) pack_cols_batched<uint16_t, kFmtNib><<<g, 256, 0, s>>>(d_jobs, d_start, njobs);
    else pack_cols_batched<uint8_t, kFmtNib><<<g, 256, 0, s>>>(d_jobs, d_start, njobs);
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

int64_t recombine_job_blocks(const RecombineParams& p) {
  return p.blocked ? ceil_div(p.m, 128) * p.tiles_n : ceil_div(p.m * ceil_div(ceil_div(p.n, 32), 4), 256);
}

cudaError_t launch_recombine_batched(const RecombineParams* d_jobs, const int64_t* d_start, int njobs,
                                     int64_t blocks, int elem_bytes, cudaStream_t s, int64_t* launches) {
  if (njobs <= 0 || blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (elem_bytes == 2) recombine_batched<uint16_t><<<(unsigned)blocks, 256, 0, s>>>(d_jobs, d_start, njobs);
  else recombine_batched<uint8_t><<<(unsigned)blocks, 256, 0, s>>>(d_jobs, d_start, njobs);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_recombine(const RecombineParams& p, cudaStream_t s, int64_t* launches) {
  const int64_t g = recombine_job_blocks(p);
  if (p.r > 64 || (reinterpret_cast<uintptr_t>(p.P) & 15u) != 0) return cudaErrorInvalidValue;
  if (p.blocked ? (p.tcols < 16 || p.tcols > 256 || p.tcols % 16 != 0 || p.bstride % 4 != 0 ||
                   p.tiles_n * p.tcols < p.n)
                : p.ldw % 4 != 0)
    return cudaErrorInvalidValue;
  switch (p.e) {
    case 2: return launch_pdl(recombine_kernel<uint8_t, 2>, g, 256, s, launches, p.pdl != 0, p);
    case 3: return launch_pdl(recombine_kernel<uint8_t, 3>, g, 256, s, launches, p.pdl != 0, p);
    case 4: return launch_pdl(recombine_kernel<uint8_t, 4>, g, 256, s, launches, p.pdl != 0, p);
    case 5: return launch_pdl(recombine_kernel<uint8_t, 5>, g, 256, s, launches, p.pdl != 0, p);
    case 6: return launch_pdl(recombine_kernel<uint8_t, 6>, g, 256, s, launches, p.pdl != 0, p);
    case 7: return launch_pdl(recombine_kernel<uint8_t, 7>, g, 256, s, launches, p.pdl != 0, p);
    case 8: return launch_pdl(recombine_kernel<uint8_t, 8>, g, 256, s, launches, p.pdl != 0, p);
    case 9: return launch_pdl(recombine_kernel<uint16_t, 9>, g, 256, s, launches, p.pdl != 0, p);
    case 10: return launch_pdl(recombine_kernel<uint16_t, 10>, g, 256, s, launches, p.pdl != 0, p);
  }
  return cudaErrorInvalidValue;
}

}  // namespace m4rie
