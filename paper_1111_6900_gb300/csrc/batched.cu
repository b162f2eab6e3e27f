// Many independent GF(2^e) products in one persistent tcgen05 launch,
// recorded once into a CUDA graph and replayed.
//
// A plan holds, in one device allocation, the per-product tables (tensor maps
// and tile ranges of the GEMM jobs, operand-plane jobs) and the operand planes
// of every product.  Its graph is: memsets for k = 0 products, one batched
// plane kernel for the rows of the A operands and one for the columns of the B
// operands (read through shared-memory tiles, no transpose), and one
// persistent GEMM over all tiles of all products, and one batched
// recombination for the products that take the Karatsuba schedule.  A
// product takes the alpha^j-B schedule (e^2 GF(2) products concatenated
// along K, the reduction folded into B, elements written by the GEMM) or the
// Karatsuba-like one (r < e^2 products whose parities the GEMM writes as
// blocked planes, recombined into elements by the last kernel).  The plan is cached in the context and reused while the
// caller passes the same descriptor array contents (same pointers, sizes and
// fields); a different array rebuilds it.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "context.h"
#include "schedule.h"

namespace m4rie {

struct BatchedPlan {
  std::vector<m4rie_problem> key;
  int fmt = 0;
  void* dmem = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
  int64_t products = 0;
  // what one batch issues (device tables inside dmem)
  std::vector<int> zero;
  std::vector<size_t> zero_bytes;
  std::vector<void*> zero_ptr;
  const PackParams* pj = nullptr;
  const int64_t* ps = nullptr;
  const TcJob* tj = nullptr;
  const int* tilejob = nullptr;
  const RecombineParams* rj = nullptr;
  const int64_t* rs = nullptr;
  int pcount[4] = {}, rcount[2] = {};
  int64_t pblocks[4] = {}, rblocks[2] = {};
  int nl = 0;
  int64_t tiles = 0;
  // phase timing: events before the plane kernels, before and after the GEMM
  // and after the recombination, recorded when the plan is issued eagerly
  cudaEvent_t ev[4] = {};
};

void destroy_plan(BatchedPlan* plan) {
  if (!plan) return;
  for (cudaEvent_t e : plan->ev)
    if (e) cudaEventDestroy(e);
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->cap) cudaStreamDestroy(plan->cap);
  if (plan->dmem) cudaFree(plan->dmem);
  delete plan;
}

namespace {

struct Interval {
  uintptr_t lo, hi;  // [lo, hi)
  bool out;
};

// No output may overlap another output or any input.
bool outputs_disjoint(int count, const m4rie_problem* pr) {
  std::vector<Interval> iv;
  iv.reserve(3 * count);
  for (int i = 0; i < count; ++i) {
    const uintptr_t w = pr[i].e <= 8 ? 1 : 2;
    if (pr[i].m > 0 && pr[i].k > 0) iv.push_back({(uintptr_t)pr[i].A, (uintptr_t)pr[i].A + w * pr[i].m * pr[i].k, false});
    if (pr[i].k > 0 && pr[i].n > 0) iv.push_back({(uintptr_t)pr[i].B, (uintptr_t)pr[i].B + w * pr[i].k * pr[i].n, false});
    if (pr[i].m > 0 && pr[i].n > 0) iv.push_back({(uintptr_t)pr[i].C, (uintptr_t)pr[i].C + w * pr[i].m * pr[i].n, true});
  }
  std::sort(iv.begin(), iv.end(), [](const Interval& a, const Interval& b) { return a.lo < b.lo; });
  // sweep: the furthest-reaching interval seen so far, and the furthest-reaching output
  uintptr_t max_hi = 0, max_out_hi = 0;
  for (const Interval& x : iv) {
    if (x.out && x.lo < max_hi) return false;  // output starts inside an earlier interval
    if (!x.out && x.lo < max_out_hi) return false;  // input starts inside an earlier output
    max_hi = std::max(max_hi, x.hi);
    if (x.out) max_out_hi = std::max(max_out_hi, x.hi);
  }
  return true;
}

m4rie_status fail(m4rie_ctx* ctx, cudaError_t err, BatchedPlan* plan) {
  ctx->last_error = cudaGetErrorString(err);
  destroy_plan(plan);
  return M4RIE_ERR_CUDA;
}

struct Layout {
  int e, eb, G, BN;
  int64_t Kp, ld, ld_bytes, Mp, groups, brows;
  size_t a_off, b_off;  // offsets into the workspace
  // Karatsuba jobs: r GF(2) products, B planes of Np rows each, parity
  // planes (blocked, p_plane words each) at p_off
  bool kara = false;
  int r = 1;
  int64_t Np = 0, p_plane = 0;
  size_t p_off = 0;
  Schedule sc;
};

// Schedule of one product of a batch: the context's setting, else the rule
// measured on GB300 (Karatsuba once its products are fewer than e^2 and the
// product is large enough for the saved MMA work to outweigh the extra A
// planes and the recombination pass).
bool use_karatsuba(const m4rie_ctx* ctx, const m4rie_problem& p, int r) {
  if (r >= p.e * p.e) return false;
  const int sched = ctx->batched_force ? ctx->batched_force : ctx->batched_sched;
  if (sched == M4RIE_SCHED_ALPHA_B) return false;
  if (sched == M4RIE_SCHED_KARATSUBA) return true;
  const TuneEntry& t = ctx->btuned[p.e][shape_class(p.m, p.n, p.k)];
  if (t.sched) return t.sched == M4RIE_SCHED_KARATSUBA;
  return p.e >= ctx->batched_kara_min_e && (double)p.m * p.n * p.k >= ctx->batched_kara_min_mnk;
}

// Tile width of one product of a batch: kTileWide, the widest tile of its
// form (alpha^j-B: e G columns with G = tc_group(e); Karatsuba: 240 for FP4,
// 256 for FP8), or kTileNarrow, the narrowest tile that still covers the
// product's columns in one tile where they are fewer; the tuner's measured
// choice for the class, else wide for alpha^j-B and narrow for Karatsuba.
enum { kTileDefault = 0, kTileWide = 1, kTileNarrow = 2 };
// the wide Karatsuba tile: FP4 MMAs of N = 240 (its scale factors take TMEM
// columns 240..255), FP8 ones of N = 256
constexpr int kara_wide(int fmt) { return fmt == kFmtNib ? 240 : 256; }
int tile_choice(const m4rie_ctx* ctx, const m4rie_problem& p, bool kara) {
  if (ctx->batched_force_width) return ctx->batched_force_width;
  const TuneEntry& t = ctx->btuned[p.e][shape_class(p.m, p.n, p.k)];
  if (t.sched && t.group_m) return t.group_m;
  return kara ? kTileNarrow : kTileWide;
}

}  // namespace

namespace {
// The launches of one batch on stream st: memsets of the k = 0 products, the
// plane kernels, the persistent GEMM, the recombinations; with `timed`, the
// plan's events around the three phases.
cudaError_t issue_plan(m4rie_ctx* ctx, BatchedPlan* plan, cudaStream_t st, bool timed, int64_t* launches) {
  cudaError_t rec = timed ? cudaEventRecord(plan->ev[0], st) : cudaSuccess;
  for (size_t i = 0; i < plan->zero_ptr.size() && rec == cudaSuccess; ++i)
    rec = cudaMemsetAsync(plan->zero_ptr[i], 0, plan->zero_bytes[i], st);
  int jo = 0, so = 0;
  for (int grp = 0; grp < 4; ++grp) {
    if (rec == cudaSuccess)
      rec = grp >= 2 ? launch_cols_batched(plan->pj + jo, plan->ps + so, plan->pcount[grp], plan->pblocks[grp],
                                           plan->fmt, (grp & 1) ? 2 : 1, st, launches)
                     : launch_pack_batched(plan->pj + jo, plan->ps + so, plan->pcount[grp], plan->pblocks[grp],
                                           plan->fmt, (grp & 1) ? 2 : 1, st, launches);
    jo += plan->pcount[grp];
    so += plan->pcount[grp] + 1;
  }
  if (rec == cudaSuccess && timed) rec = cudaEventRecord(plan->ev[1], st);
  if (rec == cudaSuccess)
    rec = launch_tc_batched(plan->fmt, plan->tj, plan->tilejob, plan->nl, plan->tiles, ctx->d_status,
                            ctx->wait_limit_ns, ctx->num_sms, st, launches);
  if (rec == cudaSuccess && timed) rec = cudaEventRecord(plan->ev[2], st);
  if (rec == cudaSuccess)
    rec = launch_recombine_batched(plan->rj, plan->rs, plan->rcount[0], plan->rblocks[0], 1, st, launches);
  if (rec == cudaSuccess)
    rec = launch_recombine_batched(plan->rj + plan->rcount[0], plan->rs + plan->rcount[0] + 1, plan->rcount[1],
                                   plan->rblocks[1], 2, st, launches);
  if (rec == cudaSuccess && timed) rec = cudaEventRecord(plan->ev[3], st);
  return rec;
}

// One batch of a recorded plan: a graph replay, or, with phase timing on, the
// same launches issued eagerly between the plan's events (which the context's
// phase times then read).
m4rie_status run_plan(m4rie_ctx* ctx, BatchedPlan* plan) {
  cudaError_t err = cudaSuccess;
  if (ctx->timing) {
    for (int i = 0; i < 4 && err == cudaSuccess; ++i)
      if (!plan->ev[i]) err = cudaEventCreate(&plan->ev[i]);
    int64_t launches = 0;
    if (err == cudaSuccess) err = issue_plan(ctx, plan, ctx->stream, true, &launches);
    if (err == cudaSuccess) {
      for (int ph = 0; ph < 3; ++ph) ctx->ev_pending.push_back({ph, {plan->ev[ph], plan->ev[ph + 1]}});
      ctx->timed_products += plan->products;
      ctx->launches += launches;
    }
  } else {
    err = cudaGraphLaunch(plan->exec, ctx->stream);
    if (err == cudaSuccess) ctx->launches += plan->launches;
  }
  if (err != cudaSuccess) {
    ctx->last_error = cudaGetErrorString(err);
    return M4RIE_ERR_CUDA;
  }
  return M4RIE_OK;
}
}  // namespace

m4rie_status run_batched(m4rie_ctx* ctx, int count, const m4rie_problem* pr, int fmt) {
  // cached plan for the same descriptors?
  if (ctx->plan && ctx->plan->fmt == fmt && (int)ctx->plan->key.size() == count &&
      std::memcmp(ctx->plan->key.data(), pr, sizeof(m4rie_problem) * (size_t)count) == 0)
    return run_plan(ctx, ctx->plan);
  if (!outputs_disjoint(count, pr)) return M4RIE_ERR_ALIAS;
  destroy_plan(ctx->plan);
  ctx->plan = nullptr;
  cudaError_t err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) {
    ctx->last_error = cudaGetErrorString(err);
    return M4RIE_ERR_CUDA;
  }

  BatchedPlan* plan = new BatchedPlan();
  plan->key.assign(pr, pr + count);
  plan->fmt = fmt;
  const int bits = fmt == kFmtNib ? 4 : 8;
  const uint32_t one = fmt == kFmtNib ? 0x2u : 0x38u;

  // ---- layouts and workspace offsets
  std::vector<int> live;  // products with m, n, k > 0
  std::vector<int> zero;  // mul products with k == 0 (C = 0)
  std::vector<Layout> lay(count);
  size_t ws = 0;
  for (int i = 0; i < count; ++i) {
    const m4rie_problem& p = pr[i];
    if (p.m == 0 || p.n == 0) continue;
    if (p.k == 0) {
      if (!p.accumulate) zero.push_back(i);
      continue;
    }
    Layout& L = lay[i];
    L.e = p.e;
    L.eb = p.e <= 8 ? 1 : 2;
    L.Kp = round_up(p.k, 128);
    L.Mp = round_up(p.m, 128);
    if (karatsuba_schedule(p.e, p.f, &L.sc) && use_karatsuba(ctx, p, L.sc.r)) {
      // r products L_p(A) R_p(B); tiles as wide as the columns need, at most
      // 240 (FP4) or 256 (FP8), in whole 16-column groups of the parity blocks
      L.kara = true;
      L.r = L.sc.r;
      const int wide = kara_wide(fmt);
      L.BN = tile_choice(ctx, p, true) == kTileNarrow ? (int)std::min<int64_t>(wide, round_up(p.n, 16)) : wide;
      L.G = L.BN;
      L.ld = L.Kp;
      L.ld_bytes = L.ld * bits / 8;
      L.Np = round_up(p.n, L.BN);
      L.groups = L.Np / L.BN;
      L.brows = L.Np;
      L.p_plane = (L.Mp / 128) * L.groups * 1024;
      L.a_off = ws;
      ws += round_up((int64_t)L.r * L.Mp * L.ld_bytes, 1024);
      L.b_off = ws;
      ws += round_up((int64_t)L.r * L.Np * L.ld_bytes, 1024);
      L.p_off = ws;
      ws += round_up((int64_t)L.r * L.p_plane * 4, 1024);
    } else {
      L.G = tc_group(p.e, fmt);
      if (tile_choice(ctx, p, false) == kTileNarrow) {
        // the fewest elements per tile that cover n, with e G a multiple of 16
        const int step = 16 / std::gcd(p.e, 16);
        L.G = (int)std::min<int64_t>(L.G, round_up(p.n, step));
      }
      L.BN = p.e * L.G;
      L.ld = (int64_t)p.e * L.Kp;
      L.ld_bytes = L.ld * bits / 8;
      L.groups = ceil_div(p.n, L.G);
      L.brows = L.groups * L.BN;
      L.a_off = ws;
      ws += round_up(L.Mp * L.ld_bytes, 1024);
      L.b_off = ws;
      ws += round_up(L.brows * L.ld_bytes, 1024);
    }
    live.push_back(i);
  }
  const int nl = (int)live.size();

  // ---- device tables: GEMM jobs, plane jobs (A u8, A u16, B u8, B u16 groups)
  std::vector<TcJob> tjobs(nl);
  std::vector<PackParams> pjobs;                    // grouped: A/u8, A/u16, B/u8, B/u16
  std::vector<int64_t> pstart;                      // block starts per group, each followed by the total
  int pcount[4] = {0, 0, 0, 0};
  int64_t pblocks[4] = {0, 0, 0, 0};

  const size_t off_tjobs = 0;
  const size_t off_pjobs = round_up(sizeof(TcJob) * (size_t)std::max(nl, 1), 256);
  const size_t off_pstart = off_pjobs + round_up(sizeof(PackParams) * 2 * (size_t)std::max(nl, 1), 256);
  // tile -> job table (upper bound on the tile count: every job's tiles)
  int64_t tiles_ub = 0;
  int nkara = 0;
  for (int i : live) {
    tiles_ub += (int64_t)lay[i].r * (lay[i].Mp / 128) * lay[i].groups;
    nkara += lay[i].kara ? 1 : 0;
  }
  const size_t off_tilejob = off_pstart + round_up(sizeof(int64_t) * (2 * (size_t)nl + 4), 256);
  // recombination jobs of the Karatsuba products and their block starts
  const size_t off_rjobs = off_tilejob + round_up(sizeof(int) * (size_t)std::max<int64_t>(tiles_ub, 1), 256);
  const size_t off_rstart = off_rjobs + round_up(sizeof(RecombineParams) * (size_t)std::max(nkara, 1), 256);
  const size_t off_ws = off_rstart + round_up(sizeof(int64_t) * (2 * (size_t)nkara + 4), 1024);
  err = cudaMalloc(&plan->dmem, off_ws + ws);
  if (err != cudaSuccess) {
    cudaGetLastError();
    destroy_plan(plan);
    ctx->last_error = "batched plan allocation failed";
    return M4RIE_ERR_NOMEM;
  }
  uint8_t* dbase = static_cast<uint8_t*>(plan->dmem);
  uint8_t* wbase = dbase + off_ws;

  // GEMM jobs, longest tiles first so that the static tile order balances the SMs
  std::vector<int> order(live);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return lay[a].ld_bytes * lay[a].BN > lay[b].ld_bytes * lay[b].BN;
  });
  int64_t tiles = 0;
  for (int t = 0; t < nl; ++t) {
    const int i = order[t];
    const m4rie_problem& p = pr[i];
    const Layout& L = lay[i];
    TcJob& j = tjobs[t];
    memset(&j, 0, sizeof(j));
    if (!tc_make_map(&j.ma, wbase + L.a_off, (int64_t)L.r * L.Mp, L.ld_bytes, 128) ||
        !tc_make_map(&j.mb, wbase + L.b_off, (int64_t)L.r * L.brows, L.ld_bytes, L.BN)) {
      destroy_plan(plan);
      ctx->last_error = "tensor map encoding failed";
      return M4RIE_ERR_CUDA;
    }
    j.C = p.C;
    j.m = p.m;
    j.n = p.n;
    j.ldc = p.n;
    j.e = p.e;
    j.G = L.G;
    j.BN = L.BN;
    j.kblocks = (int)ceil_div(L.ld_bytes, 128);
    j.kc = std::max(1, ctx->tc_chunk / 128);
    j.tiles_m = (int)(L.Mp / 128);
    j.tiles_n = (int)L.groups;
    j.elem_bytes = L.eb;
    j.add = p.accumulate ? 1 : 0;
    j.emask = (1u << p.e) - 1;
    j.mode = L.kara ? 2 : 0;
    j.batch = L.r;
    j.a_brows = L.Mp;
    j.b_brows = L.brows;
    if (L.kara) {
      j.C = wbase + L.p_off;  // parity planes; the recombination writes C
      j.p_bstride = L.p_plane;
    }
    j.tile_start = tiles;
    tiles += (int64_t)L.r * j.tiles_m * j.tiles_n;
  }
  std::vector<int> tile_job((size_t)tiles);
  for (int t = 0; t < nl; ++t)
    for (int64_t x = 0; x < (int64_t)tjobs[t].batch * tjobs[t].tiles_m * tjobs[t].tiles_n; ++x)
      tile_job[tjobs[t].tile_start + x] = t;

  // plane jobs, grouped by side and element width
  for (int grp = 0; grp < 4; ++grp) {
    const bool bside = grp >= 2;
    const int want_eb = (grp & 1) ? 2 : 1;
    for (int i : live) {
      const m4rie_problem& p = pr[i];
      const Layout& L = lay[i];
      if (L.eb != want_eb) continue;
      uint16_t amask[10], bmask[100];
      if (!L.kara) alpha_b_masks(p.e, p.f, amask, bmask);
      PackParams q{};
      q.elem_bytes = L.eb;
      q.K = p.k;
      q.fmt = fmt;
      q.one = one;
      q.kb = p.e;
      q.Kp = L.Kp;
      q.ld = L.ld;
      q.emask = (1u << p.e) - 1;
      q.e = p.e;
      q.status = ctx->d_status;
      if (L.kara) {
        // r planes per side, one mask each (Section 5's operand sums)
        q.kb = 1;
        q.nb = 1;
        q.G = 1;
        q.P = L.r;
        if (!bside) {
          q.X = p.A;
          q.ldx = p.k;
          q.vec = ((uintptr_t)p.A & 15u) == 0 && (p.k * L.eb) % 16 == 0;
          q.rows = p.m;
          q.rows_p = L.Mp;
          q.bstride = L.Mp * L.Kp;
          q.out = wbase + L.a_off;
          for (int jj = 0; jj < L.r; ++jj) q.mask[jj] = L.sc.amask[jj];
        } else {
          q.X = p.B;
          q.ldx = p.n;
          q.rows = p.n;
          q.rows_p = L.Np;
          q.bstride = L.Np * L.Kp;
          q.out = wbase + L.b_off;
          for (int jj = 0; jj < L.r; ++jj) q.mask[jj] = L.sc.bmask[jj];
        }
      } else if (!bside) {
        q.X = p.A;
        q.ldx = p.k;
        q.vec = ((uintptr_t)p.A & 15u) == 0 && (p.k * L.eb) % 16 == 0;
        q.rows = p.m;
        q.rows_p = L.Mp;
        q.P = p.e;
        q.nb = 1;
        q.G = 1;
        q.out = wbase + L.a_off;
        for (int jj = 0; jj < p.e; ++jj) q.mask[jj] = amask[jj];
      } else {
        q.X = p.B;  // k x n: the plane rows are its columns
        q.ldx = p.n;
        q.rows = p.n;
        q.rows_p = L.groups * L.G;
        q.P = p.e * p.e;
        q.nb = p.e;
        q.G = L.G;
        q.emajor = 1;  // tcgen05 epilogue: slices of an element in adjacent columns
        q.out = wbase + L.b_off;
        for (int jj = 0; jj < p.e * p.e; ++jj) q.mask[jj] = bmask[jj];
      }
      if (!plane_offsets(q)) {
        destroy_plan(plan);
        return M4RIE_ERR_UNSUPPORTED;
      }
      pstart.push_back(pblocks[grp]);
      pblocks[grp] += bside ? cols_job_blocks(q) : pack_job_blocks(q);
      pjobs.push_back(q);
      ++pcount[grp];
    }
    pstart.push_back(pblocks[grp]);  // group terminator (not read by the kernel)
  }
  // recombination jobs of the Karatsuba products, bytes first, then halfwords
  std::vector<RecombineParams> rjobs;
  std::vector<int64_t> rstart;
  int rcount[2] = {0, 0};
  int64_t rblocks[2] = {0, 0};
  for (int w = 0; w < 2; ++w) {
    for (int i : live) {
      const Layout& L = lay[i];
      if (!L.kara || L.eb != w + 1) continue;
      const m4rie_problem& p = pr[i];
      RecombineParams rc{};
      rc.P = reinterpret_cast<const uint32_t*>(wbase + L.p_off);
      rc.rows_p = L.Mp;
      rc.blocked = 1;
      rc.tcols = L.BN;
      rc.tiles_n = L.groups;
      rc.bstride = L.p_plane;
      rc.r = L.r;
      rc.e = p.e;
      rc.m = p.m;
      rc.n = p.n;
      rc.C = p.C;
      rc.ldc = p.n;
      rc.elem_bytes = L.eb;
      rc.add = p.accumulate ? 1 : 0;
      rc.emask = (1u << p.e) - 1;
      rc.status = ctx->d_status;
      for (int q = 0; q < 10; ++q) rc.out_mask[q] = L.sc.out_mask[q];
      rstart.push_back(rblocks[w]);
      rblocks[w] += recombine_job_blocks(rc);
      rjobs.push_back(rc);
      ++rcount[w];
    }
    rstart.push_back(rblocks[w]);
  }
  if (nl) {
    err = cudaMemcpy(dbase + off_tjobs, tjobs.data(), sizeof(TcJob) * nl, cudaMemcpyHostToDevice);
    if (err == cudaSuccess && !rjobs.empty())
      err = cudaMemcpy(dbase + off_rjobs, rjobs.data(), sizeof(RecombineParams) * rjobs.size(), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
      err = cudaMemcpy(dbase + off_rstart, rstart.data(), sizeof(int64_t) * rstart.size(), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
      err = cudaMemcpy(dbase + off_pjobs, pjobs.data(), sizeof(PackParams) * pjobs.size(), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
      err = cudaMemcpy(dbase + off_pstart, pstart.data(), sizeof(int64_t) * pstart.size(), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
      err = cudaMemcpy(dbase + off_tilejob, tile_job.data(), sizeof(int) * tile_job.size(), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return fail(ctx, err, plan);
  }

  // ---- what the batch issues, kept in the plan so that it can be recorded
  // into the graph and, with phase timing on, issued eagerly between events
  plan->zero = zero;
  for (int i : zero) plan->zero_bytes.push_back((size_t)(pr[i].m * pr[i].n) * (pr[i].e <= 8 ? 1 : 2));
  for (int i : zero) plan->zero_ptr.push_back(pr[i].C);
  plan->pj = reinterpret_cast<const PackParams*>(dbase + off_pjobs);
  plan->ps = reinterpret_cast<const int64_t*>(dbase + off_pstart);
  plan->tj = reinterpret_cast<const TcJob*>(dbase + off_tjobs);
  plan->tilejob = reinterpret_cast<const int*>(dbase + off_tilejob);
  plan->rj = reinterpret_cast<const RecombineParams*>(dbase + off_rjobs);
  plan->rs = reinterpret_cast<const int64_t*>(dbase + off_rstart);
  for (int g = 0; g < 4; ++g) {
    plan->pcount[g] = pcount[g];
    plan->pblocks[g] = pblocks[g];
  }
  for (int w = 0; w < 2; ++w) {
    plan->rcount[w] = rcount[w];
    plan->rblocks[w] = rblocks[w];
  }
  plan->nl = nl;
  plan->tiles = tiles;
  plan->products = nl;

  // ---- record the graph on a private stream (capture is not allowed on the legacy stream)
  err = cudaStreamCreateWithFlags(&plan->cap, cudaStreamNonBlocking);
  if (err != cudaSuccess) return fail(ctx, err, plan);
  err = cudaStreamBeginCapture(plan->cap, cudaStreamCaptureModeThreadLocal);
  if (err != cudaSuccess) return fail(ctx, err, plan);
  int64_t launches = 0;
  const cudaError_t rec = issue_plan(ctx, plan, plan->cap, false, &launches);
  cudaGraph_t graph = nullptr;
  err = cudaStreamEndCapture(plan->cap, &graph);
  if (rec != cudaSuccess || err != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(ctx, rec != cudaSuccess ? rec : err, plan);
  }
  err = cudaGraphInstantiate(&plan->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (err != cudaSuccess) return fail(ctx, err, plan);
  plan->launches = launches;
  ctx->plan = plan;
  return run_plan(ctx, plan);
}

cudaError_t launch_fill_elements(void* X, int64_t count, int eb, uint32_t emask, uint64_t seed, cudaStream_t s);

}  // namespace m4rie

using namespace m4rie;

// m4rie_tune_batched: for every (e, shape class) of the batch, time up to 32
// of its products (the same shapes, synthetic elements) in the persistent
// batched launch under each schedule and keep the faster one.
extern "C" m4rie_status m4rie_tune_batched(m4rie_ctx* ctx, int count, const m4rie_problem* problems) {
  if (!ctx || count < 0 || (count && !problems)) return M4RIE_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    const m4rie_problem& p = problems[i];
    m4rie_status st = m4rie_validate(p.e, p.f, p.m, p.n, p.k, p.A, p.B, p.C);
    if (st != M4RIE_OK) return st;
  }
  if (ctx->form != M4RIE_FORM_AUTO && ctx->form != M4RIE_FORM_TC_F4 && ctx->form != M4RIE_FORM_TC_F8)
    return M4RIE_ERR_UNSUPPORTED;
  const int fmt = ctx->form == M4RIE_FORM_TC_F8 ? kFmtByte : kFmtNib;
  std::vector<std::vector<int>> cls(11 * 64);
  for (int i = 0; i < count; ++i) {
    const m4rie_problem& p = problems[i];
    if (p.m > 0 && p.n > 0 && p.k > 0) cls[p.e * 64 + shape_class(p.m, p.n, p.k)].push_back(i);
  }
  BatchedPlan* saved = ctx->plan;  // the caller's cached plan survives the tuning runs
  ctx->plan = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  m4rie_status result = err == cudaSuccess ? M4RIE_OK : M4RIE_ERR_CUDA;
  for (int key = 0; key < 11 * 64 && result == M4RIE_OK; ++key) {
    if (cls[key].empty()) continue;
    const int e = key / 64, c = key % 64;
    const int take = (int)std::min<size_t>(cls[key].size(), 32);
    const size_t eb = e <= 8 ? 1 : 2;
    size_t bytes = 0;
    for (int t = 0; t < take; ++t) {
      const m4rie_problem& p = problems[cls[key][t]];
      bytes += round_up((int64_t)((p.m * p.k + p.k * p.n + p.m * p.n) * eb), 256);
    }
    void* buf = nullptr;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) {
      cudaGetLastError();
      result = M4RIE_ERR_NOMEM;
      break;
    }
    std::vector<m4rie_problem> sub(take);
    uint8_t* at = static_cast<uint8_t*>(buf);
    for (int t = 0; t < take && err == cudaSuccess; ++t) {
      m4rie_problem q = problems[cls[key][t]];
      q.A = at;
      q.B = at + q.m * q.k * eb;
      q.C = at + (q.m * q.k + q.k * q.n) * eb;
      q.accumulate = 0;
      err = launch_fill_elements(const_cast<void*>(q.A), q.m * q.k + q.k * q.n, (int)eb, (1u << e) - 1,
                                 0x5eed0000u + (uint64_t)t, ctx->stream);
      at += round_up((int64_t)((q.m * q.k + q.k * q.n + q.m * q.n) * eb), 256);
      sub[t] = q;
    }
    Schedule sc;
    const bool kara_ok = karatsuba_schedule(e, problems[cls[key][0]].f, &sc) && sc.r < e * e;
    double best_ms = 0;
    int best = 0, best_width = 0;
    for (int cand = 0; cand < 4 && err == cudaSuccess; ++cand) {
      const int sched = cand < 2 ? M4RIE_SCHED_ALPHA_B : M4RIE_SCHED_KARATSUBA;
      const int width = cand % 2 ? kTileNarrow : kTileWide;
      if (sched == M4RIE_SCHED_KARATSUBA && !kara_ok) continue;
      // the narrow tile is another candidate only where some product of the class has fewer columns
      if (width == kTileNarrow) {
        bool differs = false;
        for (int t = 0; t < take; ++t)
          differs |= sub[t].n < (sched == M4RIE_SCHED_KARATSUBA ? kara_wide(fmt) : tc_group(e, fmt));
        if (!differs) continue;
      }
      ctx->batched_force = sched;
      ctx->batched_force_width = width;
      m4rie_status st = run_batched(ctx, take, sub.data(), fmt);  // records the plan, runs once
      for (int w = 0; w < 2 && st == M4RIE_OK; ++w) st = run_batched(ctx, take, sub.data(), fmt);
      float ms = 0;
      if (st == M4RIE_OK) err = cudaEventRecord(e0, ctx->stream);
      for (int rep = 0; rep < 5 && st == M4RIE_OK && err == cudaSuccess; ++rep) st = run_batched(ctx, take, sub.data(), fmt);
      if (st == M4RIE_OK && err == cudaSuccess) err = cudaEventRecord(e1, ctx->stream);
      if (st == M4RIE_OK && err == cudaSuccess) err = cudaEventSynchronize(e1);
      if (st == M4RIE_OK && err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      destroy_plan(ctx->plan);
      ctx->plan = nullptr;
      if (st != M4RIE_OK) {
        result = st;
        break;
      }
      if (err == cudaSuccess && (!best || ms < best_ms)) {
        best = sched;
        best_width = width;
        best_ms = ms;
      }
    }
    ctx->batched_force = 0;
    ctx->batched_force_width = 0;
    cudaStreamSynchronize(ctx->stream);
    cudaFree(buf);
    if (err != cudaSuccess) result = M4RIE_ERR_CUDA;
    if (result == M4RIE_OK && best)
      ctx->btuned[e][c] = TuneEntry{fmt == kFmtByte ? M4RIE_FORM_TC_F8 : M4RIE_FORM_TC_F4, best, best_width, best_ms / 5.0};
  }
  ctx->batched_force = 0;
  ctx->batched_force_width = 0;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  // the choices may have changed: the next batched call records a new plan
  cudaStreamSynchronize(ctx->stream);
  destroy_plan(saved);
  if (err != cudaSuccess && ctx->last_error.empty()) ctx->last_error = cudaGetErrorString(err);
  return result;
}
