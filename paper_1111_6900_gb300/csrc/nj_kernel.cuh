// Newton-John kernel template (shared by the nj_e*.cu translation units).
// Packed rows: an element takes W bits, the next length dividing 64 (2, 4, 8
// or 16), fields lowest first.  A row is a little-endian sequence of 32-bit
// words of P = 32 / W fields each; two of them make one 64-bit word of the
// public layout.
//
// Algorithm 3 adds, for every row t of B and every row r of A, the table row
// T_t[A[r][t]] into row r of C, where T_t lists the 2^e multiples of B_t
// (Algorithm 2: the e rows alpha^i B_t, then every XOR combination of them).
// A CTA keeps a tile of C (TM rows x TW packed words) in registers, four
// words (16 bytes) per lane, and walks k in chunks of KT rows of B:
//   1. build: each warp takes some rows t of the chunk; a lane packs its four
//      words of B_t, forms alpha^i B_t for i < e with a word-parallel multiply
//      by x and writes the table rows in Gray-code order (one XOR per entry);
//   2. stage the TM x KT block of A in shared memory;
//   3. use: lane (g, v) of a warp adds words 4v .. 4v + 3 of T_t[a],
//      a = A[r][t], into its g-th row of the access.  A table row is 512
//      bytes in which the 16 bytes of lane position v are stored once per row
//      group (32 / L copies for L lanes per row), so a warp's 16-byte reads
//      are conflict-free whatever the indices.
// For e >= 6 a table of 2^e rows costs more to build than a tile of 128 rows
// uses, so the scalar is split into two index fields (3+3, 4+3, 4+4, 5+4 or
// 5+5 bits): a B_t = a_lo B_t + a_hi (alpha^b0 B_t), one table each, two
// reads per entry.  Shared-memory bandwidth bounds the kernel: 16 bytes read
// per lane and entry of A (two reads with split tables).
// Small products split k over the CTAs of a cluster (up to 8); their partial
// tiles are XOR-reduced through distributed shared memory before the store.

#pragma once
#include "m4rie_internal.cuh"
#include "newton_john.h"

namespace m4rie {
namespace nj {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <int E>
struct Nj {
  static constexpr int W = E <= 2 ? 2 : E <= 4 ? 4 : E <= 8 ? 8 : 16;  // packed field width
  static constexpr int P = 32 / W;                                      // fields per 32-bit word
  static constexpr int B0 = E <= 5 ? E : (E + 1) / 2;                   // index bits of table 0
  static constexpr int B1 = E - B0;                                     // index bits of table 1 (0: none)
  static constexpr int NE = (1 << B0) + (B1 ? (1 << B1) : 0);           // table rows per row of B
  static constexpr int EB = E <= 8 ? 1 : 2;                             // element bytes
  static constexpr int AW = 4 / EB;                                     // entries of A per 32-bit word
  static constexpr int BUDGET = E == 9 ? 98304 : 65536;                 // table bytes
  static constexpr int KT0 = BUDGET / (NE * 512) < 32 ? BUDGET / (NE * 512) : 32;
  static constexpr int KT = KT0 / AW * AW;                              // rows of B per chunk
  static constexpr int PW0 = KT / AW;
  static constexpr int PW = (PW0 & 1) ? PW0 : PW0 + 1;                  // A row pitch in words (odd)
  static constexpr uint32_t LSB = W == 2 ? 0x55555555u : W == 4 ? 0x11111111u : W == 8 ? 0x01010101u : 0x00010001u;
  static constexpr uint32_t FIELDS = LSB * ((1u << E) - 1u);            // the e low bits of every field
  static constexpr uint32_t REP = EB == 1 ? 0x01010101u : 0x00010001u;  // one per element of a 32-bit word
  static constexpr uint32_t ELEMS = REP * ((1u << E) - 1u);             // the e low bits of every element
};

__device__ __forceinline__ void flag_range(int* status, bool bad) {
  if (__any_sync(0xffffffffu, bad) && bad) atomicOr(status, kStatusRange);
}

__device__ __forceinline__ uint4 xor4(uint4 a, uint4 b) { return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w); }

// x * (every field of w) in F2[x]/<f>, all fields at once: shift each field up
// by one and add f's low part where the top coefficient fell out.
template <int E>
__device__ __forceinline__ uint32_t times_x(uint32_t w, uint32_t flow) {
  constexpr uint32_t L = Nj<E>::LSB;
  const uint32_t top = (w >> (E - 1)) & L;
  const uint32_t low = w & ~(L << (E - 1));
  return (low << 1) ^ (top * flow);  // top has one bit per field, flow < 2^E: no carries
}

__host__ __device__ constexpr int ctz_c(int s) { return (s & 1) ? 0 : 1 + ctz_c(s >> 1); }

// Table rows for the combinations of M[BASE .. BASE + BITS): row gray(S) is
// row gray(S - 1) plus the basis row of the one bit in which they differ
// (unrolled at compile time, so M stays in registers).  dst steps 512 bytes a row.
template <int E, int BITS, int BASE, int S>
__device__ __forceinline__ void gray_rows(const uint4 (&M)[E], uint4* dst, uint4 val) {
  if constexpr (S < (1 << BITS)) {
    constexpr int bit = ctz_c(S);
    val = xor4(val, M[BASE + bit]);
    dst[(S ^ (S >> 1)) * 32] = val;
    gray_rows<E, BITS, BASE, S + 1>(M, dst, val);
  }
}

template <int E, int BITS, int BASE>
__device__ __forceinline__ void write_table(const uint4 (&M)[E], uint4* dst) {
  const uint4 zero = make_uint4(0, 0, 0, 0);
  dst[0] = zero;
  gray_rows<E, BITS, BASE, 1>(M, dst, zero);
}

// Elements (one byte or one uint16 each, already in range) of one 32-bit word
// of input to packed fields, and back.
template <int E>
__device__ __forceinline__ uint32_t fields_of(const uint32_t* x) {  // x: epw<E>() words of elements
  using S = Nj<E>;
  if (S::W == 8 || S::W == 16) return x[0];
  if (S::W == 4) {  // 8 bytes < 16 -> 8 nibbles
    uint32_t lo = x[0], hi = x[1];
    lo = (lo | (lo >> 4)) & 0x00FF00FFu;
    lo = (lo | (lo >> 8)) & 0x0000FFFFu;
    hi = (hi | (hi >> 4)) & 0x00FF00FFu;
    hi = (hi | (hi >> 8)) & 0x0000FFFFu;
    return lo | (hi << 16);
  }
  uint32_t w = 0;  // W == 2: 16 bytes < 4 -> 16 two-bit fields
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t y = x[q];
    y = (y | (y >> 6)) & 0x000F000Fu;
    y = (y | (y >> 12)) & 0x000000FFu;
    w |= y << (8 * q);
  }
  return w;
}

template <int E>
__device__ __forceinline__ void elements_of(uint32_t w, uint32_t* x) {
  using S = Nj<E>;
  if (S::W == 8 || S::W == 16) {
    x[0] = w;
  } else if (S::W == 4) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      uint32_t y = (w >> (16 * q)) & 0xFFFFu;
      y = (y | (y << 8)) & 0x00FF00FFu;
      y = (y | (y << 4)) & 0x0F0F0F0Fu;
      x[q] = y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t y = (w >> (8 * q)) & 0xFFu;
      y = (y | (y << 12)) & 0x000F000Fu;
      y = (y | (y << 6)) & 0x03030303u;
      x[q] = y;
    }
  }
}

// 32-bit words of elements per packed word.
template <int E>
__host__ __device__ constexpr int epw() { return Nj<E>::W == 2 ? 4 : Nj<E>::W == 4 ? 2 : 1; }

// Packed word `wc` of row t of B; fields of columns >= n are zero.
template <int E>
__device__ __forceinline__ uint32_t load_b_word(const NjParams& p, int64_t t, int64_t wc, bool& bad) {
  using S = Nj<E>;
  const int64_t c0 = wc * S::P;
  if (wc >= p.nw || c0 >= p.n) return 0;
  const int cnt = p.n - c0 < S::P ? (int)(p.n - c0) : S::P;
  if (p.packed) {
    const uint32_t w = __ldg(static_cast<const uint32_t*>(p.B) + t * p.ldb + wc);
    const uint32_t valid = cnt == S::P ? S::FIELDS : S::FIELDS & ((1u << (cnt * S::W)) - 1u);
    const uint32_t used = cnt == S::P ? 0xffffffffu : (1u << (cnt * S::W)) - 1u;
    bad |= (w & used & ~valid) != 0;
    return w & valid;
  }
  constexpr uint32_t em = (1u << E) - 1u;
  if (cnt == S::P && p.vec_b) {  // whole word, aligned: 32-bit loads of elements
    const uint32_t* src = reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(p.B) + (t * p.ldb + c0) * S::EB);
    uint32_t x[epw<E>()];
#pragma unroll
    for (int q = 0; q < epw<E>(); ++q) {
      const uint32_t r = __ldg(src + q);
      bad |= (r & ~S::ELEMS) != 0;
      x[q] = r & S::ELEMS;
    }
    return fields_of<E>(x);
  }
  uint32_t w = 0;  // edge or unaligned: element by element
#pragma unroll 1
  for (int j = 0; j < cnt; ++j) {
      const uint32_t x = S::EB == 1 ? (uint32_t)__ldg(static_cast<const uint8_t*>(p.B) + t * p.ldb + c0 + j)
                                    : (uint32_t)__ldg(static_cast<const uint16_t*>(p.B) + t * p.ldb + c0 + j);
      bad |= x > em;
      w |= (x & em) << (j * S::W);
    }
  return w;
}

// The four packed words w0 .. w0 + 3 of row t of B (one lane's 16 bytes of
// table row).  A lane's words cover 16 * epw bytes of elements, a multiple of
// 16 that starts on a 16-byte boundary when the rows do: whole words then come
// from 16-byte loads (a quarter of the 32-bit loads, each warp access touching
// as many cache lines); otherwise word by word.
template <int E>
__device__ __forceinline__ uint4 load_b_quad(const NjParams& p, int64_t t, int64_t w0, bool& bad) {
  using S = Nj<E>;
  constexpr int Q = epw<E>();
  const int64_t c0 = w0 * S::P;
  if (!p.packed && p.vec16_b && c0 + 4 * S::P <= p.n) {
    const uint4* src = reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(p.B) + (t * p.ldb + c0) * S::EB);
    uint32_t x[4 * Q];
#pragma unroll
    for (int u = 0; u < Q; ++u) {
      const uint4 v = __ldg(src + u);
      x[4 * u] = v.x;
      x[4 * u + 1] = v.y;
      x[4 * u + 2] = v.z;
      x[4 * u + 3] = v.w;
    }
#pragma unroll
    for (int q = 0; q < 4 * Q; ++q) {
      bad |= (x[q] & ~S::ELEMS) != 0;
      x[q] &= S::ELEMS;
    }
    return make_uint4(fields_of<E>(x), fields_of<E>(x + Q), fields_of<E>(x + 2 * Q), fields_of<E>(x + 3 * Q));
  }
  return make_uint4(load_b_word<E>(p, t, w0, bad), load_b_word<E>(p, t, w0 + 1, bad),
                    load_b_word<E>(p, t, w0 + 2, bad), load_b_word<E>(p, t, w0 + 3, bad));
}

// AW consecutive entries (r, t .. t + AW) of A in one 32-bit word (zero
// outside A), as staged in shared memory.
template <int E>
__device__ __forceinline__ uint32_t load_a_word(const NjParams& p, int64_t r, int64_t t, int64_t kend, bool& bad) {
  using S = Nj<E>;
  constexpr uint32_t em = (1u << E) - 1u;
  if (r >= p.m) return 0;
  if (!p.packed && p.vec_a && t + S::AW <= kend) {
    const uint32_t raw = __ldg(reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(p.A) + (r * p.lda + t) * S::EB));
    bad |= (raw & ~S::ELEMS) != 0;
    return raw & S::ELEMS;
  }
  uint32_t w = 0;
#pragma unroll
  for (int u = 0; u < S::AW; ++u) {
    if (t + u >= kend) break;
    uint32_t x;
    if (p.packed) {
      const uint32_t pw = __ldg(static_cast<const uint32_t*>(p.A) + r * p.lda + (t + u) / S::P);
      x = (pw >> (((t + u) % S::P) * S::W)) & ((1u << S::W) - 1u);
    } else if (S::EB == 1) {
      x = __ldg(static_cast<const uint8_t*>(p.A) + r * p.lda + t + u);
    } else {
      x = __ldg(static_cast<const uint16_t*>(p.A) + r * p.lda + t + u);
    }
    bad |= x > em;
    w |= (x & em) << (u * 8 * S::EB);
  }
  return w;
}

// Store packed word `wc` of row r of C (plus the old value when accumulating).
template <int E>
__device__ __forceinline__ void store_word(const NjParams& p, int64_t r, int64_t wc, uint32_t val, bool& bad) {
  using S = Nj<E>;
  constexpr uint32_t em = (1u << E) - 1u;
  const int64_t c0 = wc * S::P;
  // fields of this word inside the matrix (0 for the padding half of a 64-bit word)
  const int cnt = p.n - c0 < S::P ? (p.n > c0 ? (int)(p.n - c0) : 0) : S::P;
  if (p.packed) {
    uint32_t* dst = static_cast<uint32_t*>(p.C) + r * p.ldc + wc;
    if (p.add) {
      const uint32_t old = *dst;
      const uint32_t valid = cnt == S::P ? S::FIELDS : S::FIELDS & ((1u << (cnt * S::W)) - 1u);
      const uint32_t used = cnt == S::P ? 0xffffffffu : (1u << (cnt * S::W)) - 1u;
      bad |= (old & used & ~valid) != 0;
      val ^= old & valid;
    }
    *dst = val;
    return;
  }
  if (cnt == S::P && p.vec_c) {  // whole word, aligned: 32-bit stores of elements
    uint32_t* dst = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(p.C) + (r * p.ldc + c0) * S::EB);
    uint32_t x[epw<E>()];
    elements_of<E>(val, x);
#pragma unroll
    for (int q = 0; q < epw<E>(); ++q) {
      if (p.add) {
        const uint32_t old = dst[q];
        bad |= (old & ~S::ELEMS) != 0;
        x[q] ^= old & S::ELEMS;
      }
      dst[q] = x[q];
    }
    return;
  }
#pragma unroll 1
  for (int j = 0; j < cnt; ++j) {  // edge or unaligned: element by element
      uint32_t x = (val >> (j * S::W)) & em;
      if (S::EB == 1) {
        uint8_t* dst = static_cast<uint8_t*>(p.C) + r * p.ldc + c0 + j;
        if (p.add) {
          const uint32_t o = *dst;
          bad |= o > em;
          x ^= o & em;
        }
        *dst = (uint8_t)x;
      } else {
        uint16_t* dst = static_cast<uint16_t*>(p.C) + r * p.ldc + c0 + j;
        if (p.add) {
          const uint32_t o = *dst;
          bad |= o > em;
          x ^= o & em;
        }
        *dst = (uint16_t)x;
      }
    }
}

// Store the four packed words w0 .. w0 + 3 of row r of C (the 16 bytes of
// one lane).  Element output with whole, aligned words: every old value of
// the four words is loaded before any store, so the loads' latencies overlap
// (a store could alias a later load, so the compiler keeps them in order);
// 16-byte accesses where the rows start on 16-byte boundaries (the lane's
// 16 * epw bytes then do too), else 32-bit ones.  Otherwise word by word.
template <int E>
__device__ __forceinline__ void store_quad(const NjParams& p, int64_t r, int64_t w0, const uint4& val, bool& bad) {
  using S = Nj<E>;
  constexpr int Q = epw<E>();
  const int64_t c0 = w0 * S::P;
  if (!p.packed && p.vec16_c && c0 + 4 * S::P <= p.n) {
    uint4* dst = reinterpret_cast<uint4*>(static_cast<uint8_t*>(p.C) + (r * p.ldc + c0) * S::EB);
    uint32_t x[4 * Q];
    elements_of<E>(val.x, x);
    elements_of<E>(val.y, x + Q);
    elements_of<E>(val.z, x + 2 * Q);
    elements_of<E>(val.w, x + 3 * Q);
    if (p.add) {
      uint4 old[Q];
#pragma unroll
      for (int u = 0; u < Q; ++u) old[u] = dst[u];
#pragma unroll
      for (int u = 0; u < Q; ++u) {
        const uint32_t o[4] = {old[u].x, old[u].y, old[u].z, old[u].w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          bad |= (o[c] & ~S::ELEMS) != 0;
          x[4 * u + c] ^= o[c] & S::ELEMS;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < Q; ++u) dst[u] = make_uint4(x[4 * u], x[4 * u + 1], x[4 * u + 2], x[4 * u + 3]);
    return;
  }
  if (!p.packed && p.vec_c && c0 + 4 * S::P <= p.n) {
    uint32_t* dst = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(p.C) + (r * p.ldc + c0) * S::EB);
    uint32_t x[4][Q];
    elements_of<E>(val.x, x[0]);
    elements_of<E>(val.y, x[1]);
    elements_of<E>(val.z, x[2]);
    elements_of<E>(val.w, x[3]);
    if (p.add) {
      uint32_t old[4][Q];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < Q; ++q) old[j][q] = dst[j * Q + q];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          bad |= (old[j][q] & ~S::ELEMS) != 0;
          x[j][q] ^= old[j][q] & S::ELEMS;
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < Q; ++q) dst[j * Q + q] = x[j][q];
    return;
  }
  if (w0 < p.nw) store_word<E>(p, r, w0, val.x, bad);
  if (w0 + 1 < p.nw) store_word<E>(p, r, w0 + 1, val.y, bad);
  if (w0 + 2 < p.nw) store_word<E>(p, r, w0 + 2, val.z, bad);
  if (w0 + 3 < p.nw) store_word<E>(p, r, w0 + 3, val.w, bad);
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint4 ld_cluster4(const uint4* local, uint32_t rank) {
  uint32_t addr = (uint32_t)__cvta_generic_to_shared(local), remote;
  uint4 v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(addr), "r"(rank));
  asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(remote)
               : "memory");
  return v;
}

template <int E, int R>
__global__ void __launch_bounds__(kThreads, 2) nj_kernel(const __grid_constant__ NjParams p) {
  using S = Nj<E>;
  extern __shared__ __align__(16) uint32_t smem[];
  uint4* sT = reinterpret_cast<uint4*>(smem);  // [KT][NE][32] table rows of 512 bytes
  uint32_t* sA = smem + S::KT * S::NE * 128;   // [TM][PW] block of A
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ll = p.lg, L = 1 << ll, G = 32 >> ll;  // L lanes per row, G rows per access
  const int g = lane >> ll, v = lane & (L - 1);
  const int TM = kWarps * R * G;
  const int64_t r0 = (int64_t)blockIdx.x * TM;
  const int64_t w0 = ((int64_t)blockIdx.y * L + v) * 4;  // first of this lane's four packed words
  const int64_t kbeg = (int64_t)blockIdx.z * p.kper;
  const int64_t kend = p.k < kbeg + p.kper ? p.k : kbeg + p.kper;
  bool bad = false;
  pdl_enter();
  uint4 acc[R];
#pragma unroll
  for (int i = 0; i < R; ++i) acc[i] = make_uint4(0, 0, 0, 0);

  // Software pipeline: the B words and the A block of chunk c + 1 are read
  // into registers while chunk c's lookups run.  Build work items are (row t
  // of the chunk, table) pairs spread over the warps.
  constexpr int NT = S::B1 ? 2 : 1;
  constexpr int NBI = (S::KT * NT + kWarps - 1) / kWarps;  // build items per warp
  uint4 bq[NBI];
  uint32_t aq[S::PW0];  // a thread stages at most TM * PW0 / 256 <= PW0 words of A
  auto fetch = [&](int64_t t0) {
    const int kt = kend - t0 < S::KT ? (int)(kend - t0) : S::KT;
    const int ktw = (kt + S::AW - 1) / S::AW;
#pragma unroll
    for (int n = 0; n < NBI; ++n) {
      const int tl = (warp + kWarps * n) / NT;
      bq[n] = make_uint4(0, 0, 0, 0);
      if (tl < kt) bq[n] = load_b_quad<E>(p, t0 + tl, w0, bad);
    }
#pragma unroll
    for (int n = 0; n < S::PW0; ++n) {
      const int idx = threadIdx.x + kThreads * n;
      const int rl = idx / S::PW0, q = idx % S::PW0;
      aq[n] = (idx < TM * S::PW0 && q < ktw) ? load_a_word<E>(p, r0 + rl, t0 + q * S::AW, kend, bad) : 0u;
    }
  };
  if (kbeg < kend) fetch(kbeg);

  for (int64_t t0 = kbeg; t0 < kend; t0 += S::KT) {
    const int kt = kend - t0 < S::KT ? (int)(kend - t0) : S::KT;
    const int ktw = (kt + S::AW - 1) / S::AW;  // words of A per row in this chunk
    // 1. Algorithm 2 for the rows t0 .. t0 + ktw * AW of B (rows past kt are zero)
#pragma unroll
    for (int n = 0; n < NBI; ++n) {
      const int it = warp + kWarps * n, tl = it / NT, j = it % NT;
      if (tl < ktw * S::AW) {
        uint4 M[E];
        M[0] = bq[n];
#pragma unroll
        for (int i = 1; i < E; ++i)
          M[i] = make_uint4(times_x<E>(M[i - 1].x, p.flow), times_x<E>(M[i - 1].y, p.flow),
                            times_x<E>(M[i - 1].z, p.flow), times_x<E>(M[i - 1].w, p.flow));
        uint4* dst = sT + tl * S::NE * 32 + lane;
        if constexpr (NT == 2) {
          if (j == 0)
            write_table<E, S::B0, 0>(M, dst);
          else
            write_table<E, S::B1, S::B0>(M, dst + (1 << S::B0) * 32);
        } else {
          write_table<E, S::B0, 0>(M, dst);
        }
      }
    }
    // 2. the TM x KT block of A, AW entries per word
#pragma unroll
    for (int n = 0; n < S::PW0; ++n) {
      const int idx = threadIdx.x + kThreads * n;
      if (idx < TM * S::PW0) sA[(idx / S::PW0) * S::PW + idx % S::PW0] = aq[n];
    }
    __syncthreads();
    if (t0 + S::KT < kend) fetch(t0 + S::KT);
    // 3. Algorithm 3's inner loop: C_r += T_t[A[r][t]]
    for (int q = 0; q < ktw; ++q) {
      const uint4* Tt = sT + q * S::AW * S::NE * 32 + lane;
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const uint32_t aw = sA[((warp * R + i) * G + g) * S::PW + q];
#pragma unroll
        for (int u = 0; u < S::AW; ++u) {
          const uint32_t a = (aw >> (u * 8 * S::EB)) & (S::EB == 1 ? 0xffu : 0xffffu);
          const uint4* Tu = Tt + u * S::NE * 32;
          if (S::B1) {
            const uint4 x = Tu[(a & ((1u << S::B0) - 1u)) * 32];
            const uint4 y = Tu[((1u << S::B0) + (a >> S::B0)) * 32];
            acc[i] = xor4(acc[i], xor4(x, y));
          } else {
            acc[i] = xor4(acc[i], Tu[a * 32]);
          }
        }
      }
    }
    __syncthreads();
  }

  if (p.ks == 1) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int64_t r = r0 + (warp * R + i) * G + g;
      if (r < p.m) store_quad<E>(p, r, w0, acc[i], bad);
    }
  } else {
    // XOR the partial tiles of the cluster's CTAs (one k range each): every
    // CTA publishes its tile in shared memory, then stores its share of the
    // rows with the sum read from all of them.
    uint4* sC = reinterpret_cast<uint4*>(smem);  // [TM][L] slices of four words
#pragma unroll
    for (int i = 0; i < R; ++i) sC[((warp * R + i) * G + g) * L + v] = acc[i];
    cluster_sync_all();
    const int slices = TM * L;
    const int share = (slices + p.ks - 1) / p.ks;
    const int q0 = (int)cluster_rank() * share;
    const int q1 = q0 + share < slices ? q0 + share : slices;
    for (int q = q0 + threadIdx.x; q < q1; q += kThreads) {
      uint4 val = make_uint4(0, 0, 0, 0);
      for (int s = 0; s < p.ks; ++s) val = xor4(val, ld_cluster4(sC + q, (uint32_t)s));
      const int64_t r = r0 + (q >> ll);
      const int64_t wq = ((int64_t)blockIdx.y * L + (q & (L - 1))) * 4;
      if (r < p.m) store_quad<E>(p, r, wq, val, bad);
    }
    cluster_sync_all();  // no CTA leaves while another still reads its tile
  }
  flag_range(p.status, bad);
}

template <int E>
size_t nj_smem(int R, int lg, int ks) {
  using S = Nj<E>;
  const int G = 32 >> lg, L = 1 << lg;
  const int TM = kWarps * R * G;
  const size_t main = (size_t)S::KT * S::NE * 512 + (size_t)TM * S::PW * 4;
  const size_t red = ks > 1 ? (size_t)TM * L * 16 : 0;
  return main > red ? main : red;
}

template <int E, int R>
cudaError_t launch_er(const NjParams& p, int64_t tiles_m, int64_t tiles_n, cudaStream_t s) {
  const size_t smem = nj_smem<E>(R, p.lg, p.ks);
  auto kern = nj_kernel<E, R>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)tiles_m, (unsigned)tiles_n, (unsigned)p.ks);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (p.ks > 1) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = 1;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = (unsigned)p.ks;
    ++na;
  }
  if (p.pdl) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kern, p);
}

}  // namespace nj

// Launch of the Newton-John kernel for one field size; instantiated in
// nj_e*.cu (one translation unit per group of field sizes, compiled in
// parallel).
template <int E>
cudaError_t nj_launch(const NjParams& p, int R, int64_t tiles_m, int64_t tiles_n, cudaStream_t s) {
  using namespace nj;
  switch (R) {
    case 1: return launch_er<E, 1>(p, tiles_m, tiles_n, s);
    case 2: return launch_er<E, 2>(p, tiles_m, tiles_n, s);
    case 4: return launch_er<E, 4>(p, tiles_m, tiles_n, s);
    case 8: return launch_er<E, 8>(p, tiles_m, tiles_n, s);
    case 16: return launch_er<E, 16>(p, tiles_m, tiles_n, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace m4rie
