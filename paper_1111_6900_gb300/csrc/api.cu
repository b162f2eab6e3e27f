// Host side of the C ABI (include/m4rie_gpu.h): validation, workspace,
// schedule and form selection, kernel dispatch.
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "context.h"
#include "newton_john.h"
#include "schedule.h"

using namespace m4rie;

namespace {

m4rie_status cuda_fail(m4rie_ctx* ctx, cudaError_t err) {
  if (ctx) ctx->last_error = cudaGetErrorString(err);
  return M4RIE_ERR_CUDA;
}

int elem_bytes(int e) { return e <= 8 ? 1 : 2; }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Phase markers: mark(ctx, phase) opens a phase, mark(ctx, -1) closes it.
enum { kPhasePack = 0, kPhaseGemm = 1, kPhaseRecombine = 2 };

cudaEvent_t take_event(m4rie_ctx* ctx) {
  if (ctx->ev_next == ctx->ev_pool.size()) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
    ctx->ev_pool.push_back(ev);
  }
  return ctx->ev_pool[ctx->ev_next++];
}

struct PhaseTimer {
  m4rie_ctx* ctx;
  int phase = -1;
  cudaEvent_t start = nullptr;
  explicit PhaseTimer(m4rie_ctx* c) : ctx(c) {}
  void begin(int ph) {
    end();
    if (!ctx->timing) return;
    start = take_event(ctx);
    if (start && cudaEventRecord(start, ctx->stream) == cudaSuccess) phase = ph;
  }
  void end() {
    if (phase < 0) return;
    cudaEvent_t stop = take_event(ctx);
    if (stop && cudaEventRecord(stop, ctx->stream) == cudaSuccess) ctx->ev_pending.push_back({phase, {start, stop}});
    phase = -1;
  }
  ~PhaseTimer() { end(); }
};

bool overlaps(const void* a, size_t an, const void* b, size_t bn) {
  if (!an || !bn) return false;
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + bn && y < x + an;
}

m4rie_status check_field(int e, uint32_t f) {
  if (e < 2 || e > 10) return M4RIE_ERR_ARG;
  if (poly_degree(f) != e || !poly_irreducible(f)) return M4RIE_ERR_POLY;
  return M4RIE_OK;
}

// Bytes spanned by a rows x cols window with row stride ld (elements of w bytes).
size_t span_bytes(int64_t rows, int64_t cols, int64_t ld, size_t w) {
  return rows && cols ? (size_t)((rows - 1) * ld + cols) * w : 0;
}

// c_over_b: C may coincide with B (internal callers only; see run_gemm).
m4rie_status validate_mats(int e, uint32_t f, int64_t m, int64_t n, int64_t k, const Mats& x, bool c_over_b = false) {
  m4rie_status st = check_field(e, f);
  if (st != M4RIE_OK) return st;
  if (m < 0 || n < 0 || k < 0) return M4RIE_ERR_ARG;
  // sizes the kernels index with 32-bit block counts and 64-bit offsets
  if (m > (1ll << 31) || n > (1ll << 31) || k > (1ll << 31)) return M4RIE_ERR_ARG;
  if (x.lda < k || x.ldb < n || x.ldc < n || x.lda > (1ll << 40) || x.ldb > (1ll << 40) || x.ldc > (1ll << 40))
    return M4RIE_ERR_ARG;
  if ((m > 0 && k > 0 && !x.A) || (k > 0 && n > 0 && !x.B) || (m > 0 && n > 0 && !x.C)) return M4RIE_ERR_ARG;
  const size_t w = elem_bytes(e);
  const size_t sc = span_bytes(m, n, x.ldc, w);
  if (overlaps(x.C, sc, x.A, span_bytes(m, k, x.lda, w)) ||
      (!c_over_b && overlaps(x.C, sc, x.B, span_bytes(k, n, x.ldb, w))))
    return M4RIE_ERR_ALIAS;
  return M4RIE_OK;
}

m4rie_status validate(int e, uint32_t f, int64_t m, int64_t n, int64_t k, const void* A, const void* B,
                      const void* C) {
  return validate_mats(e, f, m, n, k, Mats{A, k, B, n, const_cast<void*>(C), n});
}

m4rie_status ensure_ws(m4rie_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return M4RIE_OK;
  cudaError_t err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err);
  if (ctx->ws) cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  size_t want = bytes + (bytes >> 3);
  if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
    cudaGetLastError();
    if (cudaMalloc(&ctx->ws, bytes) != cudaSuccess) {
      cudaGetLastError();
      ctx->ws = nullptr;
      ctx->last_error = "workspace allocation failed";
      return M4RIE_ERR_NOMEM;
    }
    want = bytes;
  }
  ctx->ws_bytes = want;
  return M4RIE_OK;
}

// AUTO choices: the autotuned entry of the shape class if there is one, else a
// fixed rule from the measurements on GB300:
//  - Newton-John tables for thin inner dimensions and small products: k <= 64;
//    k <= 128 for e >= 3 when m n >= 2^22 (rank-64 and rank-128 updates, 2-5x
//    faster than the sliced forms there, whose fixed cost per output tile
//    dominates); every product of at most 2^24 multiply-adds (2^25 for e <= 4);
//  - else tcgen05 FP4 from 2^28 field multiply-adds, below that the bit-packed
//    form; Karatsuba from 2^30.
bool newton_john_wins(int e, int64_t m, int64_t n, int64_t k) {
  const double mnk = (double)m * n * k;
  if (k <= 64) return true;
  if (e >= 3 && k <= 128 && (double)m * n >= (double)(1 << 22)) return true;
  return mnk <= (double)(1 << (e <= 4 ? 25 : 24));
}

int sliced_form(int64_t m, int64_t n, int64_t k) {
  return shape_class(m, n, k) >= 28 ? M4RIE_FORM_TC_F4 : M4RIE_FORM_POPC;
}

int resolve_form(m4rie_ctx* ctx, int e, int64_t m, int64_t n, int64_t k) {
  if (ctx->form != M4RIE_FORM_AUTO) return ctx->form;
  const TuneEntry& t = ctx->tuned[e][shape_class(m, n, k)];
  if (t.form) return t.form;
  return newton_john_wins(e, m, n, k) ? M4RIE_FORM_NEWTON_JOHN : sliced_form(m, n, k);
}

int resolve_schedule(m4rie_ctx* ctx, int e, int64_t m, int64_t n, int64_t k) {
  if (ctx->schedule != M4RIE_SCHED_AUTO) return ctx->schedule;
  const TuneEntry& t = ctx->tuned[e][shape_class(m, n, k)];
  if (t.form) return t.sched;
  return shape_class(m, n, k) >= 30 ? M4RIE_SCHED_KARATSUBA : M4RIE_SCHED_ALPHA_B;
}

int resolve_group_m(m4rie_ctx* ctx, int e, int64_t m, int64_t n, int64_t k, int tiles_m) {
  int g = ctx->group_m;
  if (ctx->form == M4RIE_FORM_AUTO) {
    const TuneEntry& t = ctx->tuned[e][shape_class(m, n, k)];
    if (t.form) g = t.group_m;
  }
  return g > 0 ? std::min(g, tiles_m) : tiles_m;
}

// tcgen05 GEMMs run 2-SM pairs on m-tile pairs (rows padded to 256) when
// the pairing adds no padded tile or m is large enough for it not to matter.
bool pair_m(const m4rie_ctx* ctx, int64_t m) {
  return ctx->cluster == 3 && m > 256 && (round_up(m, 256) == round_up(m, 128) || m >= 2048);
}

struct FormInfo {
  int fmt;
  uint32_t one;
  int bits;  // bits per plane entry
};

FormInfo form_info(int form) {
  switch (form) {
    case M4RIE_FORM_POPC: return {kFmtBit, 1, 1};
    case M4RIE_FORM_TC_F8: return {kFmtByte, 0x38, 8};
    case M4RIE_FORM_MMA_S8: return {kFmtByte, 0x01, 8};
    case M4RIE_FORM_MMA_B1: return {kFmtBit, 1, 1};
    default: return {kFmtNib, 0x2, 4};
  }
}

size_t entries_bytes(int64_t entries, int bits) { return (size_t)((entries * bits + 7) / 8); }

// ---------------------------------------------------------------- alpha^j-B
// reuse_b: the B planes in the workspace are those of this B from the previous
// call (same form, n and k): only A is sliced.  The B planes sit at the start
// of the workspace, so their place does not depend on m.
m4rie_status run_alpha_b(m4rie_ctx* ctx, int form, int e, uint32_t f, int64_t m, int64_t n, int64_t k, const Mats& x,
                         int add, bool reuse_b = false) {
  const void* A = x.A;
  const void* B = x.B;
  void* C = x.C;
  const FormInfo fi = form_info(form);
  int G;
  if (form == M4RIE_FORM_POPC) G = popc_group(e);
  else if (form == M4RIE_FORM_TC_F8 || form == M4RIE_FORM_TC_F4) G = tc_group(e, fi.fmt);
  else if (form == M4RIE_FORM_MMA_S8 || form == M4RIE_FORM_MMA_B1) G = mma_group(e);
  else return M4RIE_ERR_UNSUPPORTED;
  const bool tc = form == M4RIE_FORM_TC_F8 || form == M4RIE_FORM_TC_F4;
  const int64_t Kp = round_up(k, 128);
  const int64_t ld = (int64_t)e * Kp;
  const bool pair = tc && pair_m(ctx, m);
  const int64_t Mp = round_up(m, pair ? 256 : 128);  // CTA pairs take m-tile pairs
  const int64_t groups = ceil_div(n, G);
  const int64_t brows = groups * e * G;
  const size_t a_bytes = round_up((int64_t)entries_bytes(Mp * ld, fi.bits), 1024);
  const size_t b_bytes = round_up((int64_t)entries_bytes(brows * ld, fi.bits), 1024);
  m4rie_status st = ensure_ws(ctx, a_bytes + b_bytes);
  if (st != M4RIE_OK) return st;
  uint8_t* Bp = static_cast<uint8_t*>(ctx->ws);
  uint8_t* Ap = Bp + b_bytes;

  uint16_t amask[10], bmask[100];
  alpha_b_masks(e, f, amask, bmask);
  PackParams pa{};
  pa.X = A;
  pa.ldx = x.lda;
  pa.elem_bytes = elem_bytes(e);
  pa.rows = m;
  pa.K = k;
  pa.rows_p = Mp;
  pa.fmt = fi.fmt;
  pa.one = fi.one;
  pa.P = e;
  pa.nb = 1;
  pa.kb = e;
  pa.G = 1;
  pa.Kp = Kp;
  pa.ld = ld;
  pa.bstride = 0;
  pa.emask = (1u << e) - 1;
  pa.e = e;
  pa.vec = aligned16(A) && (x.lda * elem_bytes(e)) % 16 == 0;
  pa.out = Ap;
  pa.status = ctx->d_status;
  pa.pdl = ctx->pdl;
  for (int j = 0; j < e; ++j) pa.mask[j] = amask[j];
  PackParams pb = pa;  // columns of B (k x n) are the planes' rows
  pb.X = B;
  pb.ldx = x.ldb;
  pb.rows = n;
  pb.rows_p = groups * G;
  pb.P = e * e;
  pb.nb = e;
  pb.kb = e;
  pb.G = G;
  // the tcgen05 epilogue wants the e slices of an element in adjacent columns
  pb.emajor = (form == M4RIE_FORM_TC_F8 || form == M4RIE_FORM_TC_F4) ? 1 : 0;
  pb.out = Bp;
  for (int q = 0; q < e * e; ++q) pb.mask[q] = bmask[q];
  PhaseTimer timer(ctx);
  timer.begin(kPhasePack);
  cudaError_t err = reuse_b ? launch_pack_planes(pa, ctx->stream, &ctx->launches)
                            : launch_pack_pair(pa, pb, ctx->stream, &ctx->launches);
  if (err != cudaSuccess) return cuda_fail(ctx, err);
  timer.begin(kPhaseGemm);

  if (form == M4RIE_FORM_POPC) {
    PopcParams pp{};
    pp.A = reinterpret_cast<const uint32_t*>(Ap);
    pp.B = reinterpret_cast<const uint32_t*>(Bp);
    pp.ldw = ld / 32;
    pp.m = m;
    pp.n = n;
    pp.e = e;
    pp.C = C;
    pp.ldc = x.ldc;
    pp.elem_bytes = elem_bytes(e);
    pp.add = add;
    pp.emask = (1u << e) - 1;
    pp.status = ctx->d_status;
    pp.pdl = ctx->pdl;
    err = launch_popc_fused(pp, ctx->stream, &ctx->launches);
  } else {
    TcParams tp{};
    tp.m = m;
    tp.n = n;
    tp.e = e;
    tp.G = G;
    tp.BN = e * G;
    tp.tiles_m = (int)(Mp / 128);
    tp.tiles_n = (int)groups;
    tp.batch = 1;
    const int64_t ld_bytes = (int64_t)entries_bytes(ld, fi.bits);
    tp.kblocks = (int)ceil_div(ld_bytes, 128);
    tp.kc = std::max(1, ctx->tc_chunk / 128);
    tp.group_m = resolve_group_m(ctx, e, m, n, k, tp.tiles_m);
    tp.C = C;
    tp.ldc = x.ldc;
    tp.elem_bytes = elem_bytes(e);
    tp.add = add;
    tp.emask = (1u << e) - 1;
    tp.status = ctx->d_status;
    tp.mode = 0;
    tp.wait_limit_ns = ctx->wait_limit_ns;
    tp.f4nv = ctx->f4nv;
    tp.stall_test = ctx->stall_test;
    tp.cluster = pair ? ctx->cluster : 1;
    tp.pdl = ctx->pdl;
    if (form == M4RIE_FORM_MMA_S8 || form == M4RIE_FORM_MMA_B1)
      err = launch_mma(form == M4RIE_FORM_MMA_B1, Ap, Bp, ld_bytes, tp, ctx->stream, &ctx->launches);
    else err = launch_tc(fi.fmt, Ap, Mp, Bp, brows, ld_bytes, tp, ctx->num_sms, ctx->stream, &ctx->launches);
  }
  if (err != cudaSuccess) return cuda_fail(ctx, err);
  return M4RIE_OK;
}

// ---------------------------------------------------------------- Karatsuba
m4rie_status run_karatsuba(m4rie_ctx* ctx, int form, int e, uint32_t f, int64_t m, int64_t n, int64_t k,
                           const Mats& x, int add, bool reuse_b = false) {
  const void* A = x.A;
  const void* B = x.B;
  void* C = x.C;
  if (form != M4RIE_FORM_POPC && form != M4RIE_FORM_TC_F8 && form != M4RIE_FORM_TC_F4) return M4RIE_ERR_UNSUPPORTED;
  Schedule sc;
  if (!karatsuba_schedule(e, f, &sc)) {
    ctx->last_error = "schedule construction failed its check";
    return M4RIE_ERR_ARG;
  }
  const FormInfo fi = form_info(form);
  const int r = sc.r;
  const int64_t Kp = round_up(k, 128);
  const bool pair = form != M4RIE_FORM_POPC && pair_m(ctx, m);
  const int64_t Mp = round_up(m, pair ? 256 : 128);
  // tcgen05 on 2-SM pairs, e <= 8: the GEMM's epilogue recombines the products
  // of each output tile itself (no parity planes, no recombination kernel)
  const bool fused = form != M4RIE_FORM_POPC && pair && e <= 8 && ctx->fuse_recombine && r <= 64;
  // popc parity tiles are 128 columns; tcgen05 tiles 256 (FP8) or 240 (FP4,
  // which keeps its scale factors in TMEM columns 240..255 next to each
  // accumulator; 224 with the recombination in the epilogue, whose output
  // slices are whole 32-column words).  FP4 MMAs of N = 240 keep the tensor
  // pipe busy with one barrier wait and commit per 8 of them, N = 224 ones
  // leave it idle about 7% of the time.
  const int ntile = form == M4RIE_FORM_POPC ? 128 : (form == M4RIE_FORM_TC_F8 ? 256 : (fused ? 224 : 240));
  const int64_t Np = round_up(n, ntile);
  // parity planes: popc, rows of ldp words (whole 16-byte groups); tcgen05,
  // blocks of 128 rows x 8 words per output tile (TcParams)
  const int64_t ldp = round_up(Np / 32, 4);
  const bool blocked = form != M4RIE_FORM_POPC;
  const int64_t p_plane = blocked ? (Mp / 128) * (Np / ntile) * 1024 : Mp * ldp;  // words per plane
  const size_t a_bytes = round_up((int64_t)entries_bytes((int64_t)r * Mp * Kp, fi.bits), 1024);
  const size_t b_bytes = round_up((int64_t)entries_bytes((int64_t)r * Np * Kp, fi.bits), 1024);
  const size_t p_bytes = fused ? 0 : round_up((int64_t)r * p_plane * 4, 1024);
  m4rie_status st = ensure_ws(ctx, a_bytes + b_bytes + p_bytes);
  if (st != M4RIE_OK) return st;
  uint8_t* Bp = static_cast<uint8_t*>(ctx->ws);
  uint8_t* Ap = Bp + b_bytes;
  uint32_t* Pp = reinterpret_cast<uint32_t*>(Ap + a_bytes);

  PackParams pa{};
  pa.X = A;
  pa.ldx = x.lda;
  pa.elem_bytes = elem_bytes(e);
  pa.rows = m;
  pa.K = k;
  pa.rows_p = Mp;
  pa.fmt = fi.fmt;
  pa.one = fi.one;
  pa.P = r;
  pa.nb = 1;
  pa.kb = 1;
  pa.G = 1;
  pa.Kp = Kp;
  pa.ld = Kp;
  pa.bstride = Mp * Kp;
  pa.emask = (1u << e) - 1;
  pa.e = e;
  pa.vec = aligned16(A) && (x.lda * elem_bytes(e)) % 16 == 0;
  pa.out = Ap;
  pa.status = ctx->d_status;
  pa.pdl = ctx->pdl;
  for (int p = 0; p < r; ++p) pa.mask[p] = sc.amask[p];
  PackParams pb = pa;  // columns of B (k x n) are the planes' rows
  pb.X = B;
  pb.ldx = x.ldb;
  pb.rows = n;
  pb.rows_p = Np;
  pb.bstride = Np * Kp;
  pb.out = Bp;
  for (int p = 0; p < r; ++p) pb.mask[p] = sc.bmask[p];
  PhaseTimer timer(ctx);
  timer.begin(kPhasePack);
  cudaError_t err = reuse_b ? launch_pack_planes(pa, ctx->stream, &ctx->launches)
                            : launch_pack_pair(pa, pb, ctx->stream, &ctx->launches);
  if (err != cudaSuccess) return cuda_fail(ctx, err);
  timer.begin(kPhaseGemm);

  if (form == M4RIE_FORM_POPC) {
    PopcParams pp{};
    pp.A = reinterpret_cast<const uint32_t*>(Ap);
    pp.B = reinterpret_cast<const uint32_t*>(Bp);
    pp.ldw = Kp / 32;
    pp.m = m;
    pp.n = n;
    pp.e = e;
    pp.C = Pp;
    pp.ldc = ldp;
    pp.status = ctx->d_status;
    pp.pdl = ctx->pdl;
    pp.batch = r;
    pp.a_bstride = Mp * Kp / 32;
    pp.b_bstride = Np * Kp / 32;
    pp.c_bstride = Mp * ldp;
    err = launch_popc_parity(pp, ctx->stream, &ctx->launches);
  } else {
    TcParams tp{};
    tp.m = m;
    tp.n = n;
    tp.e = e;
    tp.G = ntile;
    tp.BN = ntile;
    tp.tiles_m = (int)(Mp / 128);
    tp.tiles_n = (int)(Np / ntile);
    tp.batch = r;
    tp.a_brows = Mp;
    tp.b_brows = Np;
    const int64_t ld_bytes = (int64_t)entries_bytes(Kp, fi.bits);
    tp.kblocks = (int)ceil_div(ld_bytes, 128);
    tp.kc = std::max(1, ctx->tc_chunk / 128);
    tp.group_m = resolve_group_m(ctx, e, m, n, k, tp.tiles_m);
    tp.C = Pp;
    tp.status = ctx->d_status;
    tp.mode = 2;
    tp.p_bstride = p_plane;
    tp.wait_limit_ns = ctx->wait_limit_ns;
    tp.f4nv = ctx->f4nv;
    tp.stall_test = ctx->stall_test;
    tp.cluster = pair ? ctx->cluster : 1;
    tp.pdl = ctx->pdl;
    if (fused) {
      tp.mode = 3;
      tp.C = C;
      tp.ldc = x.ldc;
      tp.elem_bytes = elem_bytes(e);
      tp.add = add;
      tp.emask = (1u << e) - 1;
      tp.vec_c = aligned16(C) && x.ldc % 16 == 0;
      for (int q = 0; q < r; ++q) {
        uint32_t qm = 0;
        for (int s = 0; s < e; ++s) qm |= (uint32_t)((sc.out_mask[s] >> q) & 1ull) << s;
        tp.qmask[q] = (uint8_t)qm;
      }
    }
    err = launch_tc(fi.fmt, Ap, (int64_t)r * Mp, Bp, (int64_t)r * Np, ld_bytes, tp, ctx->num_sms, ctx->stream,
                    &ctx->launches);
  }
  if (err != cudaSuccess) return cuda_fail(ctx, err);
  if (fused) return M4RIE_OK;
  timer.begin(kPhaseRecombine);
  RecombineParams rc{};
  rc.P = Pp;
  rc.ldw = ldp;
  rc.rows_p = Mp;
  rc.blocked = blocked ? 1 : 0;
  rc.tcols = ntile;
  rc.tiles_n = Np / ntile;
  rc.bstride = p_plane;
  rc.r = r;
  rc.e = e;
  rc.m = m;
  rc.n = n;
  rc.C = C;
  rc.ldc = x.ldc;
  rc.elem_bytes = elem_bytes(e);
  rc.add = add;
  rc.emask = (1u << e) - 1;
  rc.status = ctx->d_status;
  rc.pdl = ctx->pdl;
  for (int s = 0; s < 10; ++s) rc.out_mask[s] = sc.out_mask[s];
  err = launch_recombine(rc, ctx->stream, &ctx->launches);
  if (err != cudaSuccess) return cuda_fail(ctx, err);
  return M4RIE_OK;
}

// Newton-John multiplication (newton_john.cu) on element arrays or packed rows.
m4rie_status run_newton_john(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k, const Mats& x,
                             int add, bool packed) {
  PhaseTimer timer(ctx);
  timer.begin(kPhaseGemm);
  NjParams p{};
  p.A = x.A;
  p.B = x.B;
  p.C = x.C;
  // packed leading dimensions arrive in 64-bit words; the kernel indexes 32-bit words
  p.lda = packed ? 2 * x.lda : x.lda;
  p.ldb = packed ? 2 * x.ldb : x.ldb;
  p.ldc = packed ? 2 * x.ldc : x.ldc;
  p.m = m;
  p.n = n;
  p.k = k;
  p.packed = packed ? 1 : 0;
  p.add = add;
  p.flow = f & ((1u << e) - 1u);
  p.status = ctx->d_status;
  p.pdl = ctx->pdl;
  if (!packed) {
    const int w = elem_bytes(e);
    auto rows4 = [w](const void* ptr, int64_t ld) { return (reinterpret_cast<uintptr_t>(ptr) & 3u) == 0 && (ld * w) % 4 == 0; };
    p.vec_a = rows4(x.A, x.lda);
    p.vec_b = rows4(x.B, x.ldb);
    p.vec_c = rows4(x.C, x.ldc);
    p.vec16_b = aligned16(x.B) && (x.ldb * w) % 16 == 0;
    p.vec16_c = aligned16(x.C) && (x.ldc * w) % 16 == 0;
  }
  const NjPlan pl = plan_newton_john(e, m, n, k, packed, ctx->num_sms);
  cudaError_t err = launch_newton_john(e, p, pl, ctx->stream, &ctx->launches);
  return err == cudaSuccess ? M4RIE_OK : cuda_fail(ctx, err);
}

}  // namespace

namespace m4rie {

m4rie_status run_gemm(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k, const Mats& x, int add,
                      bool c_over_b) {
  return run_gemm_as(ctx, e, f, m, n, k, x, add, c_over_b, -1, -1, false);
}

m4rie_status run_gemm_as(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k, const Mats& x, int add,
                         bool c_over_b, int form_as, int sched_as, bool reuse_b) {
  if (!ctx) return M4RIE_ERR_ARG;
  m4rie_status st = validate_mats(e, f, m, n, k, x, c_over_b && !add);
  if (st != M4RIE_OK) return st;
  if (m == 0 || n == 0) return M4RIE_OK;
  if (k == 0) {
    if (add) return M4RIE_OK;
    const size_t w = elem_bytes(e);
    cudaError_t err = cudaMemset2DAsync(x.C, (size_t)x.ldc * w, 0, (size_t)n * w, (size_t)m, ctx->stream);
    return err == cudaSuccess ? M4RIE_OK : cuda_fail(ctx, err);
  }
  int form = form_as >= 0 ? form_as : resolve_form(ctx, e, m, n, k);
  // Newton-John reads B while it writes C: an in-place product (C over B)
  // takes a sliced form, which reads B only while slicing it.
  if (form == M4RIE_FORM_NEWTON_JOHN && c_over_b) form = sliced_form(m, n, k);
  const int sched = sched_as >= 0 ? sched_as : resolve_schedule(ctx, e, m, n, k);
  if (ctx->timing) ++ctx->timed_products;
  if (form == M4RIE_FORM_NEWTON_JOHN) return run_newton_john(ctx, e, f, m, n, k, x, add, false);
  if (sched == M4RIE_SCHED_KARATSUBA) return run_karatsuba(ctx, form, e, f, m, n, k, x, add, reuse_b);
  return run_alpha_b(ctx, form, e, f, m, n, k, x, add, reuse_b);
}

}  // namespace m4rie

namespace {

m4rie_status run_mul(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k, const void* A,
                     const void* B, void* C, int add) {
  return run_gemm(ctx, e, f, m, n, k, Mats{A, k, B, n, C, n}, add);
}

}  // namespace

extern "C" {

m4rie_status m4rie_create(m4rie_ctx** out, void* stream) {
  if (!out) return M4RIE_ERR_ARG;
  *out = nullptr;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return M4RIE_ERR_CUDA;
  m4rie_ctx* ctx = new m4rie_ctx();
  ctx->stream = static_cast<cudaStream_t>(stream);
  ctx->device = dev;
  err = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (err == cudaSuccess) err = cudaMalloc(&ctx->d_status, sizeof(int));
  if (err == cudaSuccess) err = cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) {
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
    return M4RIE_ERR_CUDA;
  }
  // counts per chunk stay below 2^23 (FP32-exact, and the epilogue's parity trick needs x < 2^23):
  // a chunk holds at most 2 * tc_chunk FP4 entries
  if (const char* s = getenv("M4RIE_TC_CHUNK")) ctx->tc_chunk = std::min(std::max(128, atoi(s)), 1 << 21);
  if (const char* s = getenv("M4RIE_F4_KIND")) ctx->f4nv = strcmp(s, "nvf4") == 0 ? 1 : 0;
  if (const char* s = getenv("M4RIE_TC_CLUSTER")) ctx->cluster = atoi(s) == 1 ? 1 : 3;
  if (const char* s = getenv("M4RIE_PDL")) ctx->pdl = atoi(s) != 0;
  if (const char* s = getenv("M4RIE_FUSE_RECOMBINE")) ctx->fuse_recombine = atoi(s) != 0;
  if (const char* s = getenv("M4RIE_IO_PANELS")) ctx->io_panels = std::min(std::max(1, atoi(s)), kIoPanelsMax);
  if (const char* s = getenv("M4RIE_BATCHED_SCHED"))
    ctx->batched_sched = strcmp(s, "alpha_b") == 0 ? M4RIE_SCHED_ALPHA_B
                         : strcmp(s, "karatsuba") == 0 ? M4RIE_SCHED_KARATSUBA : M4RIE_SCHED_AUTO;
  if (const char* s = getenv("M4RIE_BATCHED_KARA_MIN_E")) ctx->batched_kara_min_e = atoi(s);
  if (const char* s = getenv("M4RIE_BATCHED_KARA_MIN_MNK")) ctx->batched_kara_min_mnk = atof(s);
  if (const char* s = getenv("M4RIE_ZERO_COPY")) ctx->zero_copy = atoi(s) != 0;
  if (const char* s = getenv("M4RIE_TUNE_CACHE")) m4rie_tune_load(ctx, s);  // a missing file is not an error
  *out = ctx;
  return M4RIE_OK;
}

void m4rie_destroy(m4rie_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->io) cudaFree(ctx->io);
  if (ctx->d_status) cudaFree(ctx->d_status);
  destroy_trsm_graph(ctx->trsm_graph);
  if (ctx->tws) cudaFree(ctx->tws);
  if (ctx->ews) cudaFree(ctx->ews);
  if (ctx->ews_host) cudaFreeHost(ctx->ews_host);
  if (ctx->d_gf) cudaFree(ctx->d_gf);
  for (cudaEvent_t ev : ctx->io_ev)
    if (ev) cudaEventDestroy(ev);
  if (ctx->s_in) cudaStreamDestroy(ctx->s_in);
  if (ctx->s_out) cudaStreamDestroy(ctx->s_out);
  for (cudaEvent_t ev : ctx->ech_ev)
    if (ev) cudaEventDestroy(ev);
  if (ctx->ech_side) cudaStreamDestroy(ctx->ech_side);
  if (ctx->ech_po_host) cudaFreeHost(ctx->ech_po_host);
  for (cudaEvent_t ev : ctx->ev_pool) cudaEventDestroy(ev);
  destroy_plan(ctx->plan);
  delete ctx;
}

m4rie_status m4rie_set_form(m4rie_ctx* ctx, int form) {
  if (!ctx || form < M4RIE_FORM_AUTO || form > M4RIE_FORM_NEWTON_JOHN) return M4RIE_ERR_ARG;
  ctx->form = form;
  return M4RIE_OK;
}

m4rie_status m4rie_set_schedule(m4rie_ctx* ctx, int schedule) {
  if (!ctx || schedule < M4RIE_SCHED_AUTO || schedule > M4RIE_SCHED_KARATSUBA) return M4RIE_ERR_ARG;
  ctx->schedule = schedule;
  return M4RIE_OK;
}

m4rie_status m4rie_mul(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k, const void* A,
                       const void* B, void* C) {
  return run_mul(ctx, e, f, m, n, k, A, B, C, 0);
}

m4rie_status m4rie_addmul(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k, const void* A,
                          const void* B, void* C) {
  return run_mul(ctx, e, f, m, n, k, A, B, C, 1);
}

m4rie_status m4rie_gemm(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k, const void* A,
                        int64_t lda, const void* B, int64_t ldb, void* C, int64_t ldc, int accumulate) {
  return run_gemm(ctx, e, f, m, n, k, Mats{A, lda, B, ldb, C, ldc}, accumulate ? 1 : 0);
}

namespace {

// Device address of a pinned, device-mapped host buffer (nullptr otherwise:
// pageable memory, or a host allocation the driver does not map).
void* mapped_host(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// The copy streams and events of the pipelined host-buffer products (created
// once per context; non-blocking, so they order against the context's stream
// through events only).
m4rie_status io_streams(m4rie_ctx* ctx) {
  if (ctx->s_in) return M4RIE_OK;
  cudaError_t err = cudaStreamCreateWithFlags(&ctx->s_in, cudaStreamNonBlocking);
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&ctx->s_out, cudaStreamNonBlocking);
  for (int i = 0; i < 2 * kIoPanelsMax && err == cudaSuccess; ++i)
    err = cudaEventCreateWithFlags(&ctx->io_ev[i], cudaEventDisableTiming);
  return err == cudaSuccess ? M4RIE_OK : cuda_fail(ctx, err);
}

}  // namespace

m4rie_status m4rie_mul_host(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k, const void* hA,
                            const void* hB, void* hC, int accumulate) {
  if (!ctx) return M4RIE_ERR_ARG;
  m4rie_status st = validate(e, f, m, n, k, hA, hB, hC);
  if (st != M4RIE_OK) return st;
  const size_t w = elem_bytes(e);
  const double total = (double)(m * k + k * n + (accumulate ? 2 : 1) * m * n) * (double)w;
  if (ctx->zero_copy && m > 0 && n > 0 && k > 0 && total <= (double)(8 << 20)) {
    // Small products on pinned buffers the GPU can address: the kernels read
    // A and B and write C in host memory directly (over the CPU-GPU link), no
    // staging copies.  (Large ones stage: the copy engines move about 200 GB/s
    // each way, more than these kernels' host accesses.)
    void* dA = mapped_host(hA);
    void* dB = mapped_host(hB);
    void* dC = mapped_host(hC);
    if (dA && dB && dC) {
      st = run_mul(ctx, e, f, m, n, k, dA, dB, dC, accumulate);
      if (st != M4RIE_OK) return st;
      const cudaError_t err = cudaStreamSynchronize(ctx->stream);
      return err == cudaSuccess ? M4RIE_OK : cuda_fail(ctx, err);
    }
  }
  const size_t sa = round_up((int64_t)(m * k * w), 256), sb = round_up((int64_t)(k * n * w), 256);
  const size_t sc = round_up((int64_t)(m * n * w), 256);
  if (sa + sb + sc > ctx->io_bytes) {
    cudaError_t err = cudaStreamSynchronize(ctx->stream);
    if (err != cudaSuccess) return cuda_fail(ctx, err);
    if (ctx->io) cudaFree(ctx->io);
    ctx->io = nullptr;
    ctx->io_bytes = 0;
    if (cudaMalloc(&ctx->io, sa + sb + sc) != cudaSuccess) {
      cudaGetLastError();
      return M4RIE_ERR_NOMEM;
    }
    ctx->io_bytes = sa + sb + sc;
  }
  uint8_t* dA = static_cast<uint8_t*>(ctx->io);
  uint8_t* dB = dA + sa;
  uint8_t* dC = dB + sb;
  cudaError_t err = cudaSuccess;
  if (m >= 1024 && total >= (double)(32 << 20)) {
    // Row panels: the copies of the next panels of A (and C) in, and of the
    // finished panels of C out, overlap the products of the others.  B is
    // copied and sliced once; every panel takes the form and schedule chosen
    // for the whole product, so that the later panels reuse its planes.
    if ((st = io_streams(ctx)) != M4RIE_OK) return st;
    const int P = ctx->io_panels;
    const int64_t mp = round_up(ceil_div(m, P), 256);
    const int form = resolve_form(ctx, e, m, n, k), sched = resolve_schedule(ctx, e, m, n, k);
    const uint8_t* hA8 = static_cast<const uint8_t*>(hA);
    uint8_t* hC8 = static_cast<uint8_t*>(hC);
    err = cudaMemcpyAsync(dB, hB, k * n * w, cudaMemcpyHostToDevice, ctx->s_in);
    int np = 0;
    for (int p = 0; p < P && err == cudaSuccess; ++p) {
      const int64_t r0 = p * mp, rows = std::min(m, r0 + mp) - r0;
      if (rows <= 0) break;
      err = cudaMemcpyAsync(dA + r0 * k * w, hA8 + r0 * k * w, rows * k * w, cudaMemcpyHostToDevice, ctx->s_in);
      if (err == cudaSuccess && accumulate)
        err = cudaMemcpyAsync(dC + r0 * n * w, hC8 + r0 * n * w, rows * n * w, cudaMemcpyHostToDevice, ctx->s_in);
      if (err == cudaSuccess) err = cudaEventRecord(ctx->io_ev[p], ctx->s_in);
      ++np;
    }
    if (err != cudaSuccess) return cuda_fail(ctx, err);
    for (int p = 0; p < np; ++p) {
      const int64_t r0 = p * mp, rows = std::min(m, r0 + mp) - r0;
      if ((err = cudaStreamWaitEvent(ctx->stream, ctx->io_ev[p], 0)) != cudaSuccess) return cuda_fail(ctx, err);
      st = run_gemm_as(ctx, e, f, rows, n, k, Mats{dA + r0 * k * w, k, dB, n, dC + r0 * n * w, n}, accumulate, false,
                       form, sched, p > 0);
      if (st != M4RIE_OK) return st;
      if ((err = cudaEventRecord(ctx->io_ev[P + p], ctx->stream)) != cudaSuccess ||
          (err = cudaStreamWaitEvent(ctx->s_out, ctx->io_ev[P + p], 0)) != cudaSuccess ||
          (err = cudaMemcpyAsync(hC8 + r0 * n * w, dC + r0 * n * w, rows * n * w, cudaMemcpyDeviceToHost,
                                 ctx->s_out)) != cudaSuccess)
        return cuda_fail(ctx, err);
    }
    err = cudaStreamSynchronize(ctx->s_out);
    return err == cudaSuccess ? M4RIE_OK : cuda_fail(ctx, err);
  }
  if (m > 0 && k > 0) err = cudaMemcpyAsync(dA, hA, m * k * w, cudaMemcpyHostToDevice, ctx->stream);
  if (err == cudaSuccess && k > 0 && n > 0)
    err = cudaMemcpyAsync(dB, hB, k * n * w, cudaMemcpyHostToDevice, ctx->stream);
  if (err == cudaSuccess && accumulate && m > 0 && n > 0)
    err = cudaMemcpyAsync(dC, hC, m * n * w, cudaMemcpyHostToDevice, ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err);
  st = run_mul(ctx, e, f, m, n, k, m > 0 && k > 0 ? dA : nullptr, k > 0 && n > 0 ? dB : nullptr,
               m > 0 && n > 0 ? dC : nullptr, accumulate);
  if (st != M4RIE_OK) return st;
  if (m > 0 && n > 0) err = cudaMemcpyAsync(hC, dC, m * n * w, cudaMemcpyDeviceToHost, ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  return err == cudaSuccess ? M4RIE_OK : cuda_fail(ctx, err);
}

m4rie_status m4rie_pack(m4rie_ctx* ctx, int e, int64_t rows, int64_t cols, const void* elems, uint64_t* slices,
                        int64_t ld_words) {
  if (!ctx || e < 2 || e > 10 || rows < 0 || cols < 0) return M4RIE_ERR_ARG;
  if (ld_words < (cols + 63) / 64) return M4RIE_ERR_ARG;
  if (rows > 0 && cols > 0 && (!elems || !slices)) return M4RIE_ERR_ARG;
  if (rows > 0 && ld_words > 0 && !slices) return M4RIE_ERR_ARG;
  if (overlaps(slices, (size_t)(e * rows * ld_words) * 8, elems, (size_t)(rows * cols) * elem_bytes(e)))
    return M4RIE_ERR_ALIAS;
  if (rows == 0 || ld_words == 0) return M4RIE_OK;
  cudaError_t err = launch_slice(e, rows, cols, elems, slices, ld_words, ctx->d_status, ctx->stream, &ctx->launches);
  return err == cudaSuccess ? M4RIE_OK : cuda_fail(ctx, err);
}

m4rie_status m4rie_unpack(m4rie_ctx* ctx, int e, int64_t rows, int64_t cols, const uint64_t* slices, int64_t ld_words,
                          void* elems) {
  if (!ctx || e < 2 || e > 10 || rows < 0 || cols < 0) return M4RIE_ERR_ARG;
  if (ld_words < (cols + 63) / 64) return M4RIE_ERR_ARG;
  if (rows > 0 && cols > 0 && (!elems || !slices)) return M4RIE_ERR_ARG;
  if (overlaps(slices, (size_t)(e * rows * ld_words) * 8, elems, (size_t)(rows * cols) * elem_bytes(e)))
    return M4RIE_ERR_ALIAS;
  if (rows == 0 || cols == 0) return M4RIE_OK;
  cudaError_t err = launch_cling(e, rows, cols, slices, ld_words, elems, ctx->stream, &ctx->launches);
  return err == cudaSuccess ? M4RIE_OK : cuda_fail(ctx, err);
}

m4rie_status m4rie_mul_batched(m4rie_ctx* ctx, int count, const m4rie_problem* problems) {
  if (!ctx || count < 0 || (count && !problems)) return M4RIE_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    const m4rie_problem& p = problems[i];
    m4rie_status st = validate(p.e, p.f, p.m, p.n, p.k, p.A, p.B, p.C);
    if (st != M4RIE_OK) return st;
  }
  if (count == 0) return M4RIE_OK;
  // The persistent batched launch uses the tcgen05 forms (FP4 unless FP8 is
  // requested); the CUDA-core, INT8, b1 and Newton-John forms run the products
  // one by one.
  if (ctx->form == M4RIE_FORM_POPC || ctx->form == M4RIE_FORM_MMA_S8 || ctx->form == M4RIE_FORM_MMA_B1 ||
      ctx->form == M4RIE_FORM_NEWTON_JOHN) {
    for (int i = 0; i < count; ++i) {
      const m4rie_problem& p = problems[i];
      m4rie_status st = run_mul(ctx, p.e, p.f, p.m, p.n, p.k, p.A, p.B, p.C, p.accumulate ? 1 : 0);
      if (st != M4RIE_OK) return st;
    }
    return M4RIE_OK;
  }
  return run_batched(ctx, count, problems, ctx->form == M4RIE_FORM_TC_F8 ? kFmtByte : kFmtNib);
}

int m4rie_packed_width(int e) { return e < 2 || e > 10 ? 0 : packed_width(e); }

m4rie_status m4rie_to_packed(m4rie_ctx* ctx, int e, int64_t rows, int64_t cols, const void* elems, int64_t lde,
                             uint64_t* words, int64_t ld_words) {
  if (!ctx || e < 2 || e > 10 || rows < 0 || cols < 0 || lde < cols || rows > (1ll << 31) || cols > (1ll << 31))
    return M4RIE_ERR_ARG;
  const int per = 64 / packed_width(e);
  if (ld_words < ceil_div(cols, per) || ld_words > (1ll << 40)) return M4RIE_ERR_ARG;
  if (rows == 0 || ld_words == 0) return M4RIE_OK;
  if ((cols && !elems) || !words) return M4RIE_ERR_ARG;
  if (overlaps(words, span_bytes(rows, ld_words, ld_words, 8), elems, span_bytes(rows, cols, lde, elem_bytes(e))))
    return M4RIE_ERR_ALIAS;
  cudaError_t err = launch_to_packed(e, rows, cols, elems, lde, reinterpret_cast<uint32_t*>(words), 2 * ld_words,
                                     ctx->d_status, ctx->stream, &ctx->launches);
  return err == cudaSuccess ? M4RIE_OK : cuda_fail(ctx, err);
}

m4rie_status m4rie_from_packed(m4rie_ctx* ctx, int e, int64_t rows, int64_t cols, const uint64_t* words,
                               int64_t ld_words, void* elems, int64_t lde) {
  if (!ctx || e < 2 || e > 10 || rows < 0 || cols < 0 || lde < cols || rows > (1ll << 31) || cols > (1ll << 31))
    return M4RIE_ERR_ARG;
  const int per = 64 / packed_width(e);
  if (ld_words < ceil_div(cols, per) || ld_words > (1ll << 40)) return M4RIE_ERR_ARG;
  if (rows == 0 || cols == 0) return M4RIE_OK;
  if (!elems || !words) return M4RIE_ERR_ARG;
  if (overlaps(words, span_bytes(rows, ld_words, ld_words, 8), elems, span_bytes(rows, cols, lde, elem_bytes(e))))
    return M4RIE_ERR_ALIAS;
  cudaError_t err = launch_from_packed(e, rows, cols, reinterpret_cast<const uint32_t*>(words), 2 * ld_words, elems,
                                       lde, ctx->stream, &ctx->launches);
  return err == cudaSuccess ? M4RIE_OK : cuda_fail(ctx, err);
}

m4rie_status m4rie_mul_packed(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k,
                              const uint64_t* A, int64_t lda, const uint64_t* B, int64_t ldb, uint64_t* C,
                              int64_t ldc, int accumulate) {
  if (!ctx) return M4RIE_ERR_ARG;
  m4rie_status st = check_field(e, f);
  if (st != M4RIE_OK) return st;
  if (m < 0 || n < 0 || k < 0 || m > (1ll << 31) || n > (1ll << 31) || k > (1ll << 31)) return M4RIE_ERR_ARG;
  const int per = 64 / packed_width(e);
  const int64_t kw = ceil_div(k, per), nw = ceil_div(n, per);
  if (lda < kw || ldb < nw || ldc < nw || lda > (1ll << 40) || ldb > (1ll << 40) || ldc > (1ll << 40))
    return M4RIE_ERR_ARG;
  if ((m > 0 && k > 0 && !A) || (k > 0 && n > 0 && !B) || (m > 0 && n > 0 && !C)) return M4RIE_ERR_ARG;
  const size_t sc = span_bytes(m, nw, ldc, 8);
  if (overlaps(C, sc, A, span_bytes(m, kw, lda, 8)) || overlaps(C, sc, B, span_bytes(k, nw, ldb, 8)))
    return M4RIE_ERR_ALIAS;
  if (m == 0 || n == 0) return M4RIE_OK;
  if (k == 0) {
    if (accumulate) return M4RIE_OK;
    cudaError_t err = cudaMemset2DAsync(C, (size_t)ldc * 8, 0, (size_t)nw * 8, (size_t)m, ctx->stream);
    return err == cudaSuccess ? M4RIE_OK : cuda_fail(ctx, err);
  }
  if (ctx->timing) ++ctx->timed_products;
  return run_newton_john(ctx, e, f, m, n, k, Mats{A, lda, B, ldb, C, ldc}, accumulate ? 1 : 0, true);
}

m4rie_status m4rie_get_device_status(m4rie_ctx* ctx) {
  if (!ctx) return M4RIE_ERR_ARG;
  int h = 0;
  cudaError_t err = cudaMemcpyAsync(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err);
  if (h & kStatusTimeout) return M4RIE_ERR_TIMEOUT;
  if (h & kStatusSingular) return M4RIE_ERR_SINGULAR;
  if (h & kStatusRange) return M4RIE_ERR_RANGE;
  return M4RIE_OK;
}

int m4rie_schedule_products(int e, uint32_t f, int schedule) {
  m4rie_status st = check_field(e, f);
  if (st != M4RIE_OK) return -(int)st;
  if (schedule == M4RIE_SCHED_ALPHA_B) return e * e;
  if (schedule == M4RIE_SCHED_KARATSUBA) {
    Schedule sc;
    if (!karatsuba_schedule(e, f, &sc)) return -(int)M4RIE_ERR_ARG;
    return sc.r;
  }
  return -(int)M4RIE_ERR_ARG;
}

m4rie_status m4rie_validate(int e, uint32_t f, int64_t m, int64_t n, int64_t k, const void* A, const void* B,
                            const void* C) {
  return validate(e, f, m, n, k, A, B, C);
}

int m4rie_schedule_masks(int e, uint32_t f, int schedule, int cap, uint16_t* amask, uint16_t* bmask,
                         uint64_t* out_mask) {
  m4rie_status st = check_field(e, f);
  if (st != M4RIE_OK) return -(int)st;
  if (!amask || !bmask || !out_mask) return -(int)M4RIE_ERR_ARG;
  for (int s = 0; s < 10; ++s) out_mask[s] = 0;
  if (schedule == M4RIE_SCHED_ALPHA_B) {
    if (cap < e * e) return -(int)M4RIE_ERR_ARG;
    uint16_t am[10], bm[100];
    alpha_b_masks(e, f, am, bm);
    for (int i = 0; i < e; ++i)
      for (int j = 0; j < e; ++j) {
        const int p = i * e + j;
        amask[p] = am[j];
        bmask[p] = bm[i * e + j];
        if (e * e <= 64) out_mask[i] |= 1ull << p;
      }
    return e * e;
  }
  if (schedule == M4RIE_SCHED_KARATSUBA) {
    Schedule sc;
    if (!karatsuba_schedule(e, f, &sc)) return -(int)M4RIE_ERR_ARG;
    if (cap < sc.r) return -(int)M4RIE_ERR_ARG;
    for (int p = 0; p < sc.r; ++p) {
      amask[p] = sc.amask[p];
      bmask[p] = sc.bmask[p];
    }
    for (int s = 0; s < 10; ++s) out_mask[s] = sc.out_mask[s];
    return sc.r;
  }
  return -(int)M4RIE_ERR_ARG;
}

int m4rie_resolve_form(m4rie_ctx* ctx, int e, int64_t m, int64_t n, int64_t k) {
  if (!ctx || e < 2 || e > 10) return -(int)M4RIE_ERR_ARG;
  return resolve_form(ctx, e, m, n, k);
}

const char* m4rie_status_string(m4rie_status s) {
  switch (s) {
    case M4RIE_OK: return "ok";
    case M4RIE_ERR_ARG: return "invalid argument";
    case M4RIE_ERR_POLY: return "field polynomial does not have degree e or is reducible";
    case M4RIE_ERR_ALIAS: return "output overlaps an input";
    case M4RIE_ERR_RANGE: return "an input entry was >= 2^e (its low e bits were used)";
    case M4RIE_ERR_NOMEM: return "workspace allocation failed";
    case M4RIE_ERR_CUDA: return "CUDA error";
    case M4RIE_ERR_TIMEOUT: return "a bounded wait inside a kernel ran out";
    case M4RIE_ERR_UNSUPPORTED: return "form not available for this problem or device";
    case M4RIE_ERR_SCRATCH: return "problem too large for the fixed scratch of m4rie_mul_noalloc";
    case M4RIE_ERR_SINGULAR: return "a triangular matrix had a zero on its diagonal";
  }
  return "unknown status";
}

const char* m4rie_last_error(m4rie_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int64_t m4rie_kernel_launches(m4rie_ctx* ctx) { return ctx ? ctx->launches : 0; }

m4rie_status m4rie_enable_timing(m4rie_ctx* ctx, int on) {
  if (!ctx) return M4RIE_ERR_ARG;
  ctx->timing = on != 0;
  return M4RIE_OK;
}

m4rie_status m4rie_phase_times(m4rie_ctx* ctx, double* pack_ms, double* gemm_ms, double* recombine_ms,
                               int64_t* products, int reset) {
  if (!ctx) return M4RIE_ERR_ARG;
  cudaError_t err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err);
  for (auto& pe : ctx->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) ctx->phase_ms[pe.first] += ms;
  }
  ctx->ev_pending.clear();
  ctx->ev_next = 0;
  if (pack_ms) *pack_ms = ctx->phase_ms[kPhasePack];
  if (gemm_ms) *gemm_ms = ctx->phase_ms[kPhaseGemm];
  if (recombine_ms) *recombine_ms = ctx->phase_ms[kPhaseRecombine];
  if (products) *products = ctx->timed_products;
  if (reset) {
    ctx->phase_ms[0] = ctx->phase_ms[1] = ctx->phase_ms[2] = 0;
    ctx->timed_products = 0;
  }
  return M4RIE_OK;
}

m4rie_status m4rie_set_test_hook(m4rie_ctx* ctx, int flags) {
  if (!ctx || (flags & ~1)) return M4RIE_ERR_ARG;
  ctx->stall_test = flags & 1;
  return M4RIE_OK;
}

m4rie_status m4rie_set_wait_limit_ns(m4rie_ctx* ctx, uint64_t ns) {
  if (!ctx) return M4RIE_ERR_ARG;
  ctx->wait_limit_ns = ns;
  return M4RIE_OK;
}

}  // extern "C"
