// GF(2) slice GEMM on the tcgen05 tensor cores (sm_103a).
//
// Operands are 0/1 slice planes encoded exactly as FP8 E4M3 (1.0 = 0x38,
// kind::f8f6f4) or as FP4 E2M1 (1.0 = 0x2, kind::mxf4 / mxf4nvf4 with unit
// block scales held in tensor memory).  Each tcgen05.mma accumulates integer
// counts sum_t a_t b_t in FP32 in tensor memory.  Counts are bounded per
// accumulation chunk (kc k-blocks of 128 bytes), so every partial sum is an
// integer below 2^23 and exact; after each chunk the epilogue warps take the
// low bit (the GF(2) sum) and XOR it into per-row bit vectors.  With the
// alpha^j-B schedule the tile's columns are the e slices of G consecutive
// output elements (column c*e + i holds slice i of element c), so the
// epilogue assembles finished field elements (Section 5: product of slice
// polynomials with the reduction mod f folded into B); with the Karatsuba
// schedule it writes one parity plane per GF(2) product, or XORs the
// products of a tile into its output slices itself (mode 3).
//
// Structure: persistent, 6 warps per CTA.  Warp 0 issues TMA loads
// (128-byte swizzled tiles) into a shared-memory ring, warp 1 issues the
// MMAs into two TMEM accumulators, warps 2-5 drain TMEM.  The default runs
// 2-SM pairs (cta_group::2, M = 256): each CTA of a 2-CTA cluster loads its
// 128 rows of A and half of the B tile, the even CTA issues the MMAs for
// both and its commits release stages and accumulators in both (3 stages of
// two k-blocks each: one barrier wait and one commit per 8 MMAs).
// Single-CTA tiles (M = 128, 4 or 5 stages of one k-block) serve small m and
// the batched launch.  No TMA load is
// multicast: every CTA loads its own tiles.  Every wait is bounded by a
// global-timer limit; on expiry the CTA sets the timeout status, stops
// issuing, waits (bounded) for its copies in flight, frees TMEM and returns.
#include <algorithm>
#include <cstring>

#include "m4rie_internal.cuh"

namespace m4rie {
namespace {

constexpr int STAGES = 4;
constexpr int A_TILE = 128 * 128;  // bytes
constexpr int B_SLOT = 256 * 128;  // bytes (tile N <= 256)
// Ring depth and B slot size: 4 stages of 256-row B slots, or 5 stages of
// 224-row slots (tile N <= 224), which still fit in 227 KB of shared memory.
__host__ __device__ constexpr int b_slot(int stages) { return stages > 4 ? 224 * 128 : B_SLOT; }
// 2-SM pairs hold half of B per CTA: at most 120 rows (FP4 tiles N <= 240) or
// 128 rows (FP8, N <= 256).
__host__ __device__ constexpr int cg2_b_slot(int fmt) { return (fmt == kFmtNib ? 120 : 128) * 128; }
constexpr int ACC_COLS = 256;
constexpr int THREADS = 192;
// Bound on the waits that drain copies and MMAs already in flight when a CTA
// aborts; independent of the (possibly tiny) wait limit that triggered it.
constexpr uint64_t DRAIN_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on phase `parity`.  Returns false when the CTA is aborting.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status,
                                          uint64_t limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;  // try_wait itself suspends for a while
    if ((it & 15u) == 0) {                   // check abort and the clock every 16 tries
      if (*abort_flag) return false;
      if (gtimer() - t0 > limit_ns) {
        *abort_flag = 1;
        atomicOr(status, kStatusTimeout);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"(map), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}

// Bulk copy of `bytes` (a multiple of 16) from shared to global memory,
// tracked by this thread's bulk-async group.
// The parity planes are read back by the recombination right after the GEMM:
// they are written with an L2 evict-last hint, so that the GEMM's own stream
// of operand planes does not push them out to DRAM first.
__device__ __forceinline__ void bulk_store(void* gdst, uint32_t ssrc, uint32_t bytes) {
  uint64_t policy;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(policy));
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(gdst),
               "r"(ssrc), "r"(bytes), "l"(policy)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Wait until this thread's bulk copies have read their shared-memory sources.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Wait until this thread's bulk copies are complete.
__device__ __forceinline__ void bulk_wait() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f8f6f4: D = F32, A = B = E4M3, both K-major.
__host__ __device__ constexpr uint32_t idesc_f8(int M, int N) {
  return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor, kind::mxf4 / kind::mxf4nvf4 (block scaled): A = B
// = E2M1, both K-major, scale factors UE8M0 (mxf4) or UE4M3 (nvf4), scale-factor
// ids 0, dense K = 64, D = F32.
__host__ __device__ constexpr uint32_t idesc_f4(int M, int N, bool nv) {
  return (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | (nv ? 0u : (1u << 23)) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f8(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// D (+)= A * B with per-32-element block scales read from tensor memory
// (all scales are 2^0 here, so the products are the plain 0/1 counts).
template <bool NV>
__device__ __forceinline__ void mma_f4(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t sf,
                                       uint32_t acc) {
  if (NV)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %5, 0;\n"
        "tcgen05.mma.cta_group::1.kind::mxf4nvf4.block_scale.scale_vec::4X [%0], %1, %2, %3, [%4], [%4], p;\n}\n" ::
            "r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(sf), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %5, 0;\n"
        "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%4], p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(sf), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// ---- 2-SM (cta_group::2) forms: one MMA of M = 256 rows reads 128 rows of A
// and half of B from the shared memory of each CTA of a 2-CTA cluster and
// writes 128 accumulator rows into each CTA's tensor memory.
__device__ __forceinline__ void mma_f8_cg2(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

template <bool NV>
__device__ __forceinline__ void mma_f4_cg2(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t sf,
                                           uint32_t acc) {
  if (NV)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %5, 0;\n"
        "tcgen05.mma.cta_group::2.kind::mxf4nvf4.block_scale.scale_vec::4X [%0], %1, %2, %3, [%4], [%4], p;\n}\n" ::
            "r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(sf), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %5, 0;\n"
        "tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%4], p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(sf), "r"(acc)
        : "memory");
}

// Arrive (once the pair's MMAs issued so far complete) on the barrier at the
// same shared-memory offset in both CTAs.
__device__ __forceinline__ void mma_commit_cg2(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"((uint16_t)3)
      : "memory");
}

// TMA load into this CTA's shared memory whose byte count completes on an
// mbarrier of the CTA pair (bar: a shared::cluster address).
__device__ __forceinline__ void tma_load_2d_cg2(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(dst),
      "l"(map), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}

// The shared::cluster address of `addr` (a shared::cta address) in CTA `rank`.
__device__ __forceinline__ uint32_t mapa_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}
// Arrive without release semantics: for a hand-over whose only hazard is on
// tensor memory, whose accesses the arriving warp has already waited for
// (tcgen05.wait::ld / wait::st) and ordered by tcgen05.fence::before_thread_sync.
__device__ __forceinline__ void mbar_arrive_relaxed_cluster(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}
__device__ __forceinline__ void mbar_arrive_relaxed(uint32_t bar) {
  asm volatile("mbarrier.arrive.relaxed.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// 16 consecutive accumulator columns of this thread's lane, the low 16 bits
// of each (which hold a count's parity bit), two columns to a register:
// register i holds column 2i in bits 0..15 and column 2i + 1 in bits 16..31.
// Does not wait (tmem_wait_ld waits for every load issued before it).
__device__ __forceinline__ void tmem_ld16_packed(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.pack::16b.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tile_coords(const TcParams& p, int tile, int& b, int& tm, int& tn) {
  const int per = p.tiles_m * p.tiles_n;
  b = tile / per;
  tile -= b * per;
  const int span = p.group_m * p.tiles_n;
  const int grp = tile / span;
  const int first = grp * p.group_m;
  const int gm = min(p.tiles_m - first, p.group_m);
  const int local = tile - grp * span;
  tm = first + local % gm;
  tn = local / gm;
}

// Tile order of one CTA (pair).  Without FE: every tstep-th tile.  With FE
// (mode 3): tile u * batch + b is product b of output tile u; a pair runs the
// batch products of an output tile back to back, then moves tstep units on.
template <int FE>
__device__ __forceinline__ int first_tile(const TcParams& p, int tfirst) {
  return FE ? tfirst * p.batch : tfirst;
}
template <int FE>
__device__ __forceinline__ int next_tile(const TcParams& p, int tile, int tstep) {
  if (!FE) return tile + tstep;
  return (tile + 1) % p.batch ? tile + 1 : tile + 1 + (tstep - 1) * p.batch;
}

// FP4 only: TMEM columns [SF_COL, SF_COL + 16) hold the unit scale factors.
constexpr int SF_COL = 240;
// Every accumulator starts at 2^23 (the epilogue stores it into the columns
// it has drained before releasing them, and into both buffers at the start):
// an integer count x < 2^23 accumulated onto 2^23 in FP32 is exact and leaves
// x in the low mantissa bits, so bit 0 of the raw word is x mod 2.
constexpr uint32_t kBias = 0x4B000000u;  // 2^23 as FP32
__host__ __device__ constexpr int bias_cols(int fmt) { return fmt == kFmtNib ? SF_COL : ACC_COLS; }

// Store 2^23 into `cols` (a multiple of 16) accumulator columns from taddr on,
// for this warp's 32 lanes, and wait for the stores.
__device__ __forceinline__ void tmem_fill_bias(uint32_t taddr, int cols) {
  for (int c = 0; c < cols; c += 16)
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(
            taddr + c),
        "r"(kBias)
        : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Everything a role needs to know about one output tile.
struct TileV {
  const CUtensorMap* ma;
  const CUtensorMap* mb;
  int arow, brow;       // TMA row coordinates of the A and B tiles
  int BN, kblocks, kc;  // tile N, k-blocks, k-blocks per accumulation chunk
  int b, tm, tn;
  // epilogue
  void* C;
  int64_t m, n, ldc;
  int G, e, elem_bytes, add;
  uint32_t emask;
  int mode, tiles_n;    // epilogue mode; column tiles (blocked parity layout)
  int64_t p_bstride;    // parity mode: words between products
};

// Non-batched: one problem (or a batch of equally shaped parity products) in p.
// Batched: the tile's job comes from the tile -> job table.
// CL = 3: tile indices count pairs of m-tiles (2 tm, 2 tm + 1) handled by the
// two CTAs of a 2-SM pair, which share the B tile; `rank` picks this CTA's m-tile.
template <bool BATCHED, int CL = 1, int FE = 0>
__device__ __forceinline__ void get_tile(const TcParams& p, const TcJob* __restrict__ jobs, const CUtensorMap* tmA,
                                         const CUtensorMap* tmB, int tile, int& jc, TileV& t, int rank = 0) {
  if (!BATCHED) {
    if (FE) {
      int u0;
      tile_coords(p, tile / p.batch, u0, t.tm, t.tn);  // u0 = 0: units index the m x n tiles
      t.b = tile % p.batch;
    } else {
      tile_coords(p, tile, t.b, t.tm, t.tn);
    }
    if (CL == 3) t.tm = 2 * t.tm + rank;
    t.ma = tmA;
    t.mb = tmB;
    t.arow = (int)(t.b * p.a_brows) + t.tm * 128;
    t.brow = (int)(t.b * p.b_brows) + t.tn * p.BN;
    t.BN = p.BN;
    t.kblocks = p.kblocks;
    t.kc = p.kc;
    t.C = p.C;
    t.m = p.m;
    t.n = p.n;
    t.ldc = p.ldc;
    t.G = p.G;
    t.e = p.e;
    t.elem_bytes = p.elem_bytes;
    t.add = p.add;
    t.emask = p.emask;
    t.mode = p.mode;
    t.tiles_n = p.tiles_n;
    t.p_bstride = p.p_bstride;
  } else {
    jc = __ldg(p.tile_job + tile);
    const TcJob& j = jobs[jc];
    const int local = (int)(tile - j.tile_start);
    const int per = j.tiles_m * j.tiles_n;
    t.b = local / per;  // GF(2) product of the job (mode 2)
    const int rem = local - t.b * per;
    t.tm = rem % j.tiles_m;
    t.tn = rem / j.tiles_m;
    t.ma = &j.ma;
    t.mb = &j.mb;
    t.arow = (int)(t.b * j.a_brows) + t.tm * 128;
    t.brow = (int)(t.b * j.b_brows) + t.tn * j.BN;
    t.BN = j.BN;
    t.kblocks = j.kblocks;
    t.kc = j.kc;
    t.C = j.C;
    t.m = j.m;
    t.n = j.n;
    t.ldc = j.ldc;
    t.G = j.G;
    t.e = j.e;
    t.elem_bytes = j.elem_bytes;
    t.add = j.add;
    t.emask = j.emask;
    t.mode = j.mode;
    t.tiles_n = j.tiles_n;
    t.p_bstride = j.p_bstride;
  }
}

// BATCHED: p.batch = number of jobs, p.tiles_m = total tiles, p.tiles_n = 1;
// per-tile parameters come from jobs[].  NV (FP4 only): kind::mxf4nvf4 with
// UE4M3 scales per 16 entries instead of kind::mxf4 with UE8M0 per 32.
// CL = 1: single CTAs, M = 128.
// CL = 3 (non-batched): 2-SM MMAs (cta_group::2).  The even CTA issues MMAs of M = 256 that
// read A's 128 rows and B's half tile from each CTA's shared memory and write
// 128 accumulator rows into each CTA's tensor memory; each CTA holds only its
// half of B, so a stage is 128 rows of A and half of B and more stages fit.
// Both CTAs' copies complete on the even CTA's full barriers, its commits
// release stages and accumulators in both CTAs, and both epilogues release the
// even CTA's accumulator barriers.
// Mode 3 epilogue of one unit: row r of the output tile's columns
// tn * BN .. + BN as field elements (bytes, e <= FE <= 8) from the FE output
// slices (bit c of outs[s][c / 32] = coefficient s of column c); with
// accumulation the old values are XOR-ed in.  Returns true if an old entry
// was out of range.
template <int FE>
__device__ __forceinline__ bool store_slices(const TcParams& p, const TileV& t, int64_t r, int tn,
                                             const uint32_t (&outs)[FE][8]) {
  if (r >= t.m) return false;
  const int64_t c0 = (int64_t)tn * t.BN;
  const int ncols = t.n - c0 < t.BN ? (int)(t.n - c0) : t.BN;
  uint8_t* dst = static_cast<uint8_t*>(t.C) + r * t.ldc + c0;
  const uint32_t rep = 0x01010101u * t.emask;
  bool bad = false;
  // Four elements (columns 32 w + 4 q .. + 3) as one word of bytes: spread four
  // bits of each slice to the low bits of four bytes.  Every index is a
  // compile-time constant, so outs stays in registers.
  auto quad = [&](int w, int q) {
    uint32_t v = 0;
#pragma unroll
    for (int s = 0; s < FE; ++s) v |= ((((outs[s][w] >> (4 * q)) & 0xFu) * 0x00204081u) & 0x01010101u) << s;
    return v;
  };
  if (ncols == t.BN && p.vec_c) {
    uint4* d4 = reinterpret_cast<uint4*>(dst);
#pragma unroll
    for (int w0 = 0; w0 < 8; w0 += 2) {  // 64 columns per round: four 16-byte stores, old values loaded first
      uint4 old[4];
      if (t.add) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (16 * (2 * w0 + u) < t.BN) old[u] = d4[2 * w0 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int w = w0 + (u >> 1), q0 = 4 * (u & 1);
        if (16 * (2 * w0 + u) >= t.BN) break;
        uint4 v = make_uint4(quad(w, q0), quad(w, q0 + 1), quad(w, q0 + 2), quad(w, q0 + 3));
        if (t.add) {
          bad |= ((old[u].x | old[u].y | old[u].z | old[u].w) & ~rep) != 0;
          v.x ^= old[u].x & rep;
          v.y ^= old[u].y & rep;
          v.z ^= old[u].z & rep;
          v.w ^= old[u].w & rep;
        }
        d4[2 * w0 + u] = v;
      }
    }
    return bad;
  }
#pragma unroll
  for (int w = 0; w < 8; ++w)  // ragged or unaligned: byte by byte
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (32 * w + 4 * q >= ncols) continue;
      const uint32_t v = quad(w, q);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int c = 32 * w + 4 * q + i;
        if (c >= ncols) break;
        uint32_t x = (v >> (8 * i)) & 0xFFu;
        if (t.add) {
          const uint32_t o = dst[c];
          bad |= o > t.emask;
          x ^= o & t.emask;
        }
        dst[c] = (uint8_t)x;
      }
    }
  return bad;
}

template <int FMT, bool BATCHED, bool NV = false, int CL = 1, int STAGES = 4, int FE = 0, int KPS = 1>
__global__ void __launch_bounds__(THREADS, 1)
    tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ TcParams p, const TcJob* __restrict__ jobs) {
  constexpr bool CG2 = CL == 3;
  constexpr int CLN = CL == 1 ? 1 : 2;  // CTAs per cluster
  constexpr int B_SLOT = CG2 ? cg2_b_slot(FMT) : b_slot(STAGES);
  constexpr int NBAR = (2 * STAGES + 6 + 1) & ~1;  // barrier words, even
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // CG2 keeps the B slots first, so that every B-operand read of a stage,
  // even one past its half tile, stays inside this CTA's allocation
  // A stage holds KPS k-blocks: KPS A tiles and KPS B slots.
  uint8_t* sA = CG2 ? smem + STAGES * KPS * B_SLOT : smem;
  uint8_t* sB = CG2 ? smem : smem + STAGES * KPS * A_TILE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * KPS * (A_TILE + B_SLOT));
  // bars: full[STAGES], empty[STAGES], tfull[2], tempty[2], drain, never
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  uint32_t* sbits = tmem_slot + 4;  // [4 warps][32 rows][9 words] (8 bit words + a zero sentinel)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * STAGES), tempty0 = smem_u32(bars + 2 * STAGES + 2);
  const uint32_t drain = smem_u32(bars + 2 * STAGES + 4);
  const uint32_t never = smem_u32(bars + 2 * STAGES + 5);  // test hook: nothing arrives on it

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      // released by the MMA commits (CG2: the even CTA's, signalled in both CTAs)
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, CG2 ? 8 : 4);  // one arrival per epilogue warp (CG2: of both CTAs)
    }
    mbar_init(drain, 1);
    mbar_init(never, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!BATCHED) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
    }
  }
  if (warp == 1) {
    if (CG2) {
      // one warp of each CTA of the pair allocates collectively
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(2 * ACC_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(2 * ACC_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t crank = CLN == 2 ? cluster_rank() : 0;
  if (CLN == 2) cluster_sync();  // the peer's barriers are initialised before anything lands in them
  const uint32_t tmem = *tmem_slot;
  if (warp >= 2) {  // both accumulators start at 2^23 (each epilogue warp owns 32 TMEM lanes)
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
    tmem_fill_bias(tmem + lanes, bias_cols(FMT));
    tmem_fill_bias(tmem + lanes + ACC_COLS, bias_cols(FMT));
  }
  if (FMT == kFmtNib) {
    // Unit block-scale factors (UE8M0 0x7F = 2^0) for every lane, written by
    // the four epilogue warps (each owns 32 TMEM lanes).
    if (warp >= 2) {
      uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + SF_COL;
      const uint32_t v = NV ? 0x38383838u : 0x7F7F7F7Fu;  // 1.0 as UE4M3 / UE8M0
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
          "r"(v)
          : "memory");
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  // CG2: the even CTA's MMAs write the peer's accumulators (and read its scale factors)
  if (CG2) cluster_sync();
  const int total = BATCHED ? p.tiles_m : p.batch * p.tiles_m * p.tiles_n;
  const uint64_t lim = p.wait_limit_ns;
  // tile loop: every CTA (CL = 1) or every CTA pair (CL = 3) takes every
  // (gridDim.x / CLN)-th tile
  const int tfirst = blockIdx.x / CLN, tstep = gridDim.x / CLN;
  // everything above overlaps the previous kernel's tail; no role touches
  // global memory before that kernel (the operand planes' producer) is done
  pdl_enter();

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int stage = 0, jc = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0, issued_parity = 0;
      bool ok = true;
      for (int tile = first_tile<FE>(p, tfirst); tile < total && ok; tile = next_tile<FE>(p, tile, tstep)) {
        TileV t;
        get_tile<BATCHED, CL, FE>(p, jobs, &tmA, &tmB, tile, jc, t, crank);
        if (BATCHED && tile + (int)gridDim.x < total) {
          // fetch the next tile's tensor maps into the TMA descriptor cache early
          const TcJob& nj = jobs[__ldg(p.tile_job + tile + gridDim.x)];
          asm volatile("prefetch.tensormap [%0];" ::"l"(&nj.ma) : "memory");
          asm volatile("prefetch.tensormap [%0];" ::"l"(&nj.mb) : "memory");
        }
        // bytes of one k-block (CG2: the even CTA's full barrier counts both CTAs' bytes)
        const uint32_t bytes = (CG2 ? 2 * A_TILE : A_TILE) + (uint32_t)t.BN * 128;
        // stages of up to KPS k-blocks, never across an accumulation chunk
        // (the MMA warp walks the same steps)
        for (int kb0 = 0; kb0 < t.kblocks && ok; kb0 += t.kc) {
          const int kb1 = min(kb0 + t.kc, t.kblocks);
          for (int kb = kb0; kb < kb1; kb += KPS) {
            const int nk = min(KPS, kb1 - kb);
            if (!mbar_wait(empty0 + 8 * stage, phase ^ 1, abort_flag, p.status, lim)) {
              ok = false;
              break;
            }
            const uint32_t fb = full0 + 8 * stage;
            uint8_t* a_dst = sA + stage * KPS * A_TILE;
            uint8_t* b_dst = sB + stage * KPS * B_SLOT;
            if (CG2) {
              const uint32_t fb_even = mapa_rank(fb, 0);
              if (crank == 0) mbar_expect_tx(fb, bytes * nk);
              for (int h = 0; h < nk; ++h) {
                tma_load_2d_cg2(smem_u32(a_dst + h * A_TILE), t.ma, fb_even, (kb + h) * 128, t.arow);
                tma_load_2d_cg2(smem_u32(b_dst + h * B_SLOT), t.mb, fb_even, (kb + h) * 128,
                                t.brow + (int)crank * (t.BN / 2));
              }
            } else {
              mbar_expect_tx(fb, bytes * nk);
              for (int h = 0; h < nk; ++h) {
                tma_load_2d(smem_u32(a_dst + h * A_TILE), t.ma, fb, (kb + h) * 128, t.arow);
                tma_load_2d(smem_u32(b_dst + h * B_SLOT), t.mb, fb, (kb + h) * 128, t.brow);
              }
            }
            issued_mask |= 1u << stage;
            issued_parity = (issued_parity & ~(1u << stage)) | (phase << stage);
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1;
            }
          }
        }
      }
      if (!ok) {
        // Aborting: wait (bounded) for the copies this thread issued.  The odd
        // CTA of a CG2 pair cannot observe its copies (they complete on the
        // even CTA's barriers, which the even CTA drains); it waits 50 us.
        if (CG2 && crank != 0) {
          const uint64_t t0 = gtimer();
          while (gtimer() - t0 < 50000ull) {
          }
        } else {
          for (int s = 0; s < STAGES; ++s)
            if (issued_mask >> s & 1u) {
              const uint64_t t0 = gtimer();
              while (!mbar_try(full0 + 8 * s, (issued_parity >> s) & 1u) && gtimer() - t0 < DRAIN_NS) {
              }
            }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      const uint32_t sf = tmem + SF_COL;
      const uint64_t sda0 = sdesc(smem_u32(sA)), sdb0 = sdesc(smem_u32(sB));
      int stage = 0, jc = 0;
      uint32_t phase = 0;
      int chunk = 0;
      bool ok = true;
      // CG2: only the even CTA issues MMAs (for both CTAs)
      const int my_total = CG2 && crank != 0 ? 0 : total;
      for (int tile = first_tile<FE>(p, tfirst); tile < my_total && ok; tile = next_tile<FE>(p, tile, tstep)) {
        TileV t;
        get_tile<BATCHED, CL, FE>(p, jobs, &tmA, &tmB, tile, jc, t, crank);
        constexpr int MM = CG2 ? 256 : 128;
        const uint32_t idesc = FMT == kFmtNib ? idesc_f4(MM, t.BN, NV) : idesc_f8(MM, t.BN);
        for (int kb0 = 0; kb0 < t.kblocks && ok; kb0 += t.kc) {
          const int kb1 = min(kb0 + t.kc, t.kblocks);
          const int buf = chunk & 1;
          const uint32_t tph = (chunk >> 1) & 1;
          if (!mbar_wait(tempty0 + 8 * buf, tph ^ 1, abort_flag, p.status, lim)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t d = tmem + buf * ACC_COLS;
          // One barrier wait and one commit per stage of KPS k-blocks: the
          // single issuing thread needs the MMAs of about two k-blocks (8 MMAs)
          // per wait-and-commit to keep the tensor pipe busy.
          for (int kb = kb0; kb < kb1; kb += KPS) {
            const int nk = min(KPS, kb1 - kb);
            if (!mbar_wait(full0 + 8 * stage, phase, abort_flag, p.status, lim)) {
              ok = false;
              break;
            }
            fence_after();
#pragma unroll
            for (int h = 0; h < KPS; ++h) {
              if (h < nk) {
                // descriptors of this k-block's tiles; each MMA steps 32 bytes
                // of K (32 FP8 or 64 FP4 entries; 2 in the address field)
                const uint64_t da = sda0 + (uint64_t)((stage * KPS + h) * (A_TILE >> 4));
                const uint64_t db = sdb0 + (uint64_t)((stage * KPS + h) * (B_SLOT >> 4));
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                  const uint32_t acc = 1u;  // onto the 2^23 bias
                  if (CG2) {
                    if (FMT == kFmtNib) mma_f4_cg2<NV>(d, da + 2 * k, db + 2 * k, idesc, sf, acc);
                    else mma_f8_cg2(d, da + 2 * k, db + 2 * k, idesc, acc);
                  } else {
                    if (FMT == kFmtNib) mma_f4<NV>(d, da + 2 * k, db + 2 * k, idesc, sf, acc);
                    else mma_f8(d, da + 2 * k, db + 2 * k, idesc, acc);
                  }
                }
              }
            }
            if (CG2) mma_commit_cg2(empty0 + 8 * stage);
            else mma_commit(empty0 + 8 * stage);
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1;
            }
          }
          if (!ok) break;
          if (CG2) mma_commit_cg2(tfull0 + 8 * buf);
          else mma_commit(tfull0 + 8 * buf);
          ++chunk;
        }
      }
      // Every MMA this thread issued has completed once `drain` flips; only
      // then may TMEM be freed (bounded wait, also on the abort path).  CG2:
      // the even CTA's commit flips `drain` in both CTAs.
      if (!CG2) mma_commit(drain);
      else if (crank == 0) mma_commit_cg2(drain);
      const uint64_t t0 = gtimer();
      while (!mbar_try(drain, 0) && gtimer() - t0 < DRAIN_NS) {
      }
    }
  } else {
    // ---------------- epilogue: warps 2..5, TMEM lanes 32*(warp%4) ...
    const int q = warp & 3;
    const int row = 32 * q + lane;
    uint32_t* wbits = sbits + q * 32 * 9;  // this warp's 32 rows
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    int chunk = 0, jc = 0;
    // failure-detection test: a wait that can only run out
    bool ok = !p.stall_test || __all_sync(0xffffffffu, mbar_wait(never, 0, abort_flag, p.status, lim));
    // mode 3: the output slices of this thread's row, XOR-summed over the products of a unit
    uint32_t outs[FE ? FE : 1][8];
#pragma unroll
    for (int s = 0; s < (FE ? FE : 1); ++s)
#pragma unroll
      for (int w = 0; w < 8; ++w) outs[s][w] = 0;
    for (int tile = first_tile<FE>(p, tfirst); tile < total && ok; tile = next_tile<FE>(p, tile, tstep)) {
      TileV t;
      get_tile<BATCHED, CL, FE>(p, jobs, &tmA, &tmB, tile, jc, t, crank);
      const int b = t.b, tm = t.tm, tn = t.tn;
      const int nc16 = t.BN / 16;
      uint32_t bits[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int kb0 = 0; kb0 < t.kblocks; kb0 += t.kc) {
        const int buf = chunk & 1;
        const uint32_t tph = (chunk >> 1) & 1;
        // warp-uniform decision: tcgen05.ld below needs all 32 lanes
        if (!__all_sync(0xffffffffu, mbar_wait(tfull0 + 8 * buf, tph, abort_flag, p.status, lim))) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t ta = tmem + lane_base + buf * ACC_COLS;
        // 128 columns per round: eight packed loads in flight (each round
        // trip to tensor memory costs several hundred clocks), then one wait
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          uint32_t v[8][8];
#pragma unroll
          for (int h = 0; h < 8; ++h)
            if (8 * g + h < nc16) tmem_ld16_packed(ta + 16 * (8 * g + h), v[h]);
          if (8 * g < nc16) tmem_wait_ld();
#pragma unroll
          for (int h = 0; h < 8; ++h) {
            const int c16 = 8 * g + h;
            if (c16 < nc16) {
              // parity of the count: bit 0 of 2^23 + x (kBias), i.e. bits 0
              // and 16 of a packed register; t gathers column 2i's at bit 2i
              // and column 2i + 1's at bit 16 + 2i
              uint32_t t = 0;
#pragma unroll
              for (int i = 0; i < 8; ++i) t |= (v[h][i] & 0x00010001u) << (2 * i);
              const uint32_t w = (t & 0x5555u) | ((t >> 15) & 0xAAAAu);
              bits[c16 >> 1] ^= w << (16 * (c16 & 1));
            }
          }
        }
        tmem_fill_bias(ta, bias_cols(FMT));  // the next chunk in this buffer starts at 2^23 again
        // The warp's TMEM loads and stores are complete (wait::ld, wait::st)
        // and ordered before the arrive by the tcgen05 fence, which is all the
        // MMAs that next write this buffer depend on: one lane of the warp
        // arrives, without release semantics.
        fence_before();
        __syncwarp();
        if (lane == 0) {
          if (CG2) mbar_arrive_relaxed_cluster(mapa_rank(tempty0 + 8 * buf, 0));  // the even CTA's barrier
          else mbar_arrive_relaxed(tempty0 + 8 * buf);
        }
        ++chunk;
      }
      if (!ok) continue;
      const int64_t r0 = (int64_t)tm * 128;
      if constexpr (FE > 0) {
        // Karatsuba recombination (Section 5): output slice s is the XOR of
        // the parities of the products that feed it
        const uint32_t qm = p.qmask[b];
#pragma unroll
        for (int s = 0; s < FE; ++s)
          if ((qm >> s) & 1u)
#pragma unroll
            for (int w = 0; w < 8; ++w) outs[s][w] ^= bits[w];
        if (b == p.batch - 1) {
          if (store_slices<FE>(p, t, r0 + row, tn, outs)) atomicOr(p.status, kStatusRange);
#pragma unroll
          for (int s = 0; s < FE; ++s)
#pragma unroll
            for (int w = 0; w < 8; ++w) outs[s][w] = 0;
        }
        continue;
      }
      if (t.mode == 2) {
        // Parity planes, blocked: this warp's 32 rows of the tile are 1 KB of
        // contiguous words (8 per row).  The rows go to shared memory and one
        // bulk copy writes them: scattered per-row global stores from the
        // epilogue warps measurably slowed the MMAs of the same SM.
        uint32_t* blk = static_cast<uint32_t*>(t.C) + (int64_t)b * t.p_bstride +
                        ((int64_t)tm * t.tiles_n + tn) * 1024 + 32 * q * 8;
        if (lane == 0) bulk_wait_read();  // the previous copy has read the staging rows
        __syncwarp();
        uint4* st = reinterpret_cast<uint4*>(wbits) + 2 * lane;
        st[0] = make_uint4(bits[0], bits[1], bits[2], bits[3]);
        st[1] = make_uint4(bits[4], bits[5], bits[6], bits[7]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the bulk copy
        __syncwarp();
        if (lane == 0) bulk_store(blk, smem_u32(wbits), 1024);
        continue;
      }
      // Assemble field elements.  The B planes are element-major: column
      // c*E + i holds slice i of element c of this tile, so element c is the
      // E-bit field at bit c*E of the row's bit vector.  Each warp writes its
      // own 32 rows, lanes along the elements (coalesced stores).
#pragma unroll
      for (int w = 0; w < 8; ++w) wbits[lane * 9 + w] = bits[w];
      wbits[lane * 9 + 8] = 0;  // sentinel word for the funnel shift
      __syncwarp();
      const int G = t.G, E = t.e;  // G <= 128 (tile N = e * G <= 256, e >= 2)
      const int64_t c0 = (int64_t)tn * G;
      bool bad = false;
      // A lane takes elements lane, lane + 32, lane + 64, lane + 96 of each row.
      // With accumulation, the old values of 8 rows are loaded before any of
      // them is written, so the loads' latencies overlap.
      for (int rl0 = 0; rl0 < 32; rl0 += 8) {
        uint32_t old[8][4];
        if (t.add) {
#pragma unroll
          for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int64_t r = r0 + 32 * q + rl0 + i, c = c0 + lane + 32 * u;
              old[i][u] = 0;
              if (r < t.m && lane + 32 * u < G && c < t.n)
                old[i][u] = t.elem_bytes == 1 ? (uint32_t)static_cast<const uint8_t*>(t.C)[r * t.ldc + c]
                                              : (uint32_t)static_cast<const uint16_t*>(t.C)[r * t.ldc + c];
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int rl = rl0 + i;
          const int64_t r = r0 + 32 * q + rl;
          if (r >= t.m) break;
          const uint32_t* rb = wbits + rl * 9;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int cl = lane + 32 * u;
            const int64_t c = c0 + cl;
            if (cl >= G || c >= t.n) break;
            const int pos = cl * E;
            const uint64_t pair = rb[pos >> 5] | ((uint64_t)rb[(pos >> 5) + 1] << 32);
            uint32_t val = (uint32_t)(pair >> (pos & 31)) & t.emask;
            if (t.add) {
              bad |= old[i][u] > t.emask;
              val ^= old[i][u] & t.emask;
            }
            if (t.elem_bytes == 1) static_cast<uint8_t*>(t.C)[r * t.ldc + c] = (uint8_t)val;
            else static_cast<uint16_t*>(t.C)[r * t.ldc + c] = (uint16_t)val;
          }
        }
      }
      if (bad) atomicOr(p.status, kStatusRange);
      __syncwarp();
    }
    // the parity blocks' bulk copies are complete before the CTA leaves
    if (lane == 0) bulk_wait();
    __syncwarp();
  }
  fence_before();
  __syncthreads();
  fence_after();
  // no CTA of a cluster leaves while the peer may still write into its shared
  // (CG2: or tensor) memory
  if (CLN == 2) cluster_sync();
  if (warp == 1) {
    __syncwarp();
    if (CG2)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * ACC_COLS) : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * ACC_COLS) : "memory");
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}

}  // namespace

bool tc_make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t ld_bytes, int box_rows) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)ld_bytes, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld_bytes};
  cuuint32_t box[2] = {128, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int tc_group(int e, int fmt) {
  // tile N = e * G: a multiple of 16, at most 256 (FP8) or 240 (FP4, whose
  // TMEM also holds the scale factors next to each accumulator)
  const int cap = fmt == kFmtNib ? 240 : 256;
  int best = 16;
  for (int g = 1; e * g <= cap; ++g)
    if ((e * g) % 16 == 0) best = g;
  return best;
}

size_t tc_smem_bytes(int stages = STAGES) {
  return 1024 + (size_t)stages * (A_TILE + b_slot(stages)) + 16 * 8 + 16 + 128 * 9 * 4;
}

// 2-SM pairs: 3 stages of two k-blocks each (A and half of B per k-block:
// 62 KB for FP4, 64 KB for FP8).  Stages of one k-block (7 of FP4, 6 of FP8
// fit) measured slower: the one issuing thread then waits on a barrier and
// commits after every 4 MMAs, and that bookkeeping left the tensor pipe idle
// about a quarter of the time; with 8 MMAs per wait and commit it stays busy.
constexpr int CG2_STAGES = 3, CG2_KPS = 2;
size_t tc_smem_bytes_cg2(int fmt) {
  return 1024 + (size_t)CG2_STAGES * CG2_KPS * (A_TILE + cg2_b_slot(fmt)) +
         (size_t)((2 * CG2_STAGES + 6 + 1) & ~1) * 8 + 16 + 128 * 9 * 4;
}

cudaError_t launch_tc(int fmt, const void* Aplanes, int64_t a_rows, const void* Bplanes, int64_t b_rows,
                      int64_t ld_bytes, const TcParams& p, int num_sms, cudaStream_t s, int64_t* launches) {
  if (fmt != kFmtByte && fmt != kFmtNib) return cudaErrorNotSupported;
  if (p.BN % 16 != 0 || p.BN < 16 || p.BN > (fmt == kFmtNib ? SF_COL : 256) || ld_bytes % 16 != 0)
    return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  // 2-SM pairs when the m-tiles pair up (the caller pads the planes' rows to
  // a multiple of 256 for that); each CTA loads half of the B tile
  const bool pair = p.cluster == 3 && p.tiles_m % 2 == 0 && num_sms >= 2;
  if (!tc_make_map(&ma, Aplanes, a_rows, ld_bytes, 128) ||
      !tc_make_map(&mb, Bplanes, b_rows, ld_bytes, pair ? p.BN / 2 : p.BN))
    return cudaErrorInvalidValue;
  // FP4 tiles of N <= 224 take the 5-stage ring
  const bool deep = fmt == kFmtNib && p.BN <= 224;
  const size_t smem = tc_smem_bytes(deep ? 5 : 4);
  if (p.mode == 3 && !(pair && p.e <= 8)) return cudaErrorInvalidValue;
  if (pair) {
    // 2-SM MMAs: the pair computes M = 256 rows per tile
    constexpr int S = CG2_STAGES, K2 = CG2_KPS;
    auto kernel = fmt == kFmtNib ? (p.f4nv ? tc_kernel<kFmtNib, false, true, 3, S, 0, K2>
                                           : tc_kernel<kFmtNib, false, false, 3, S, 0, K2>)
                                 : tc_kernel<kFmtByte, false, false, 3, S, 0, K2>;
    if (p.mode == 3) {
      // Karatsuba with the recombination in the epilogue: output slices for e <= 4 or e <= 8
      if (fmt == kFmtNib)
        kernel = p.e <= 4 ? (p.f4nv ? tc_kernel<kFmtNib, false, true, 3, S, 4, K2> : tc_kernel<kFmtNib, false, false, 3, S, 4, K2>)
                          : (p.f4nv ? tc_kernel<kFmtNib, false, true, 3, S, 8, K2> : tc_kernel<kFmtNib, false, false, 3, S, 8, K2>);
      else
        kernel = p.e <= 4 ? tc_kernel<kFmtByte, false, false, 3, S, 4, K2> : tc_kernel<kFmtByte, false, false, 3, S, 8, K2>;
    }
    const size_t smem2 = tc_smem_bytes_cg2(fmt);
    cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    if (err != cudaSuccess) return err;
    TcParams q = p;
    q.tiles_m = p.tiles_m / 2;
    q.group_m = std::max(1, std::min(q.tiles_m, p.group_m / 2));
    const int64_t pairs = (int64_t)q.batch * q.tiles_m * q.tiles_n;
    if (pairs > 0x7fffffffLL) return cudaErrorInvalidValue;
    const int clusters = (int)std::min<int64_t>(pairs, num_sms / 2);
    if (clusters <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * clusters);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = smem2;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = p.pdl ? 2 : 1;
    err = cudaLaunchKernelEx(&cfg, kernel, ma, mb, q, (const TcJob*)nullptr);
    if (launches) ++*launches;
    return err != cudaSuccess ? err : cudaGetLastError();
  }
  auto kernel = fmt == kFmtNib ? (deep ? (p.f4nv ? tc_kernel<kFmtNib, false, true, 1, 5>
                                                 : tc_kernel<kFmtNib, false, false, 1, 5>)
                                       : (p.f4nv ? tc_kernel<kFmtNib, false, true> : tc_kernel<kFmtNib, false, false>))
                               : tc_kernel<kFmtByte, false>;
  cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int64_t total = (int64_t)p.batch * p.tiles_m * p.tiles_n;
  if (total > 0x7fffffffLL || p.a_brows * p.batch > 0x7fffffffLL || p.b_brows * p.batch > 0x7fffffffLL)
    return cudaErrorInvalidValue;
  const int grid = total < num_sms ? (int)total : num_sms;
  if (grid <= 0) return cudaSuccess;
  err = launch_ex(kernel, dim3(grid), dim3(THREADS), smem, s, p.pdl != 0, ma, mb, p, (const TcJob*)nullptr);
  if (launches) ++*launches;
  return err != cudaSuccess ? err : cudaGetLastError();
}

cudaError_t launch_tc_batched(int fmt, const TcJob* d_jobs, const int* d_tile_job, int njobs, int64_t total_tiles,
                              int* status, uint64_t wait_limit_ns, int num_sms, cudaStream_t s, int64_t* launches) {
  if (fmt != kFmtByte && fmt != kFmtNib) return cudaErrorNotSupported;
  if (njobs <= 0 || total_tiles <= 0) return cudaSuccess;
  if (total_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  TcParams p{};
  p.batch = njobs;
  p.tiles_m = (int)total_tiles;
  p.tiles_n = 1;
  p.group_m = 1;
  p.status = status;
  p.wait_limit_ns = wait_limit_ns;
  p.tile_job = d_tile_job;
  CUtensorMap dummy;
  memset(&dummy, 0, sizeof(dummy));
  const size_t smem = tc_smem_bytes();
  auto kernel = fmt == kFmtNib ? tc_kernel<kFmtNib, true> : tc_kernel<kFmtByte, true>;
  cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int grid = total_tiles < num_sms ? (int)total_tiles : num_sms;
  kernel<<<grid, THREADS, smem, s>>>(dummy, dummy, p, d_jobs);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace m4rie
