// Many independent GF(2^e) products in one persistent tcgen05 launch,
// recorded once into a CUDA graph and replayed.
//
// A plan holds, in one device allocation, the per-product tables (tensor maps
// and tile ranges of the GEMM jobs, operand-plane jobs) and the operand planes
// of every product.  Its graph is: memsets for k = 0 products, one batched
// plane kernel for the rows of the A operands and one for the columns of the B
// operands (read through shared-memory tiles, no transpose), and one
// persistent GEMM over all tiles of all products (alpha^j-B schedule, element
// epilogue).  The plan is cached in the context and reused while the
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
};

void destroy_plan(BatchedPlan* plan) {
  if (!plan) return;
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
};

}  // namespace

m4rie_status run_batched(m4rie_ctx* ctx, int count, const m4rie_problem* pr, int fmt) {
  // cached plan for the same descriptors?
  if (ctx->plan && ctx->plan->fmt == fmt && (int)ctx->plan->key.size() == count &&
      std::memcmp(ctx->plan->key.data(), pr, sizeof(m4rie_problem) * (size_t)count) == 0) {
    cudaError_t err = cudaGraphLaunch(ctx->plan->exec, ctx->stream);
    if (err != cudaSuccess) {
      ctx->last_error = cudaGetErrorString(err);
      return M4RIE_ERR_CUDA;
    }
    ctx->launches += ctx->plan->launches;
    return M4RIE_OK;
  }
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
    L.G = tc_group(p.e, fmt);
    L.BN = p.e * L.G;
    L.Kp = round_up(p.k, 128);
    L.ld = (int64_t)p.e * L.Kp;
    L.ld_bytes = L.ld * bits / 8;
    L.Mp = round_up(p.m, 128);
    L.groups = ceil_div(p.n, L.G);
    L.brows = L.groups * L.BN;
    L.a_off = ws;
    ws += round_up(L.Mp * L.ld_bytes, 1024);
    L.b_off = ws;
    ws += round_up(L.brows * L.ld_bytes, 1024);
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
  for (int i : live) tiles_ub += (lay[i].Mp / 128) * lay[i].groups;
  const size_t off_tilejob = off_pstart + round_up(sizeof(int64_t) * (2 * (size_t)nl + 4), 256);
  const size_t off_ws = off_tilejob + round_up(sizeof(int) * (size_t)std::max<int64_t>(tiles_ub, 1), 1024);
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
    if (!tc_make_map(&j.ma, wbase + L.a_off, L.Mp, L.ld_bytes, 128) ||
        !tc_make_map(&j.mb, wbase + L.b_off, L.brows, L.ld_bytes, L.BN)) {
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
    j.tile_start = tiles;
    tiles += (int64_t)j.tiles_m * j.tiles_n;
  }
  std::vector<int> tile_job((size_t)tiles);
  for (int t = 0; t < nl; ++t)
    for (int64_t x = 0; x < (int64_t)tjobs[t].tiles_m * tjobs[t].tiles_n; ++x) tile_job[tjobs[t].tile_start + x] = t;

  // plane jobs, grouped by side and element width
  for (int grp = 0; grp < 4; ++grp) {
    const bool bside = grp >= 2;
    const int want_eb = (grp & 1) ? 2 : 1;
    for (int i : live) {
      const m4rie_problem& p = pr[i];
      const Layout& L = lay[i];
      if (L.eb != want_eb) continue;
      uint16_t amask[10], bmask[100];
      alpha_b_masks(p.e, p.f, amask, bmask);
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
      if (!bside) {
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
  if (nl) {
    err = cudaMemcpy(dbase + off_tjobs, tjobs.data(), sizeof(TcJob) * nl, cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
      err = cudaMemcpy(dbase + off_pjobs, pjobs.data(), sizeof(PackParams) * pjobs.size(), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
      err = cudaMemcpy(dbase + off_pstart, pstart.data(), sizeof(int64_t) * pstart.size(), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
      err = cudaMemcpy(dbase + off_tilejob, tile_job.data(), sizeof(int) * tile_job.size(), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return fail(ctx, err, plan);
  }

  // ---- record the graph on a private stream (capture is not allowed on the legacy stream)
  err = cudaStreamCreateWithFlags(&plan->cap, cudaStreamNonBlocking);
  if (err != cudaSuccess) return fail(ctx, err, plan);
  err = cudaStreamBeginCapture(plan->cap, cudaStreamCaptureModeThreadLocal);
  if (err != cudaSuccess) return fail(ctx, err, plan);
  int64_t launches = 0;
  cudaError_t rec = cudaSuccess;
  for (int i : zero)
    if (rec == cudaSuccess)
      rec = cudaMemsetAsync(pr[i].C, 0, (size_t)(pr[i].m * pr[i].n) * (pr[i].e <= 8 ? 1 : 2), plan->cap);
  {
    const auto* pj = reinterpret_cast<const PackParams*>(dbase + off_pjobs);
    const auto* ps = reinterpret_cast<const int64_t*>(dbase + off_pstart);
    int jo = 0, so = 0;
    for (int grp = 0; grp < 4; ++grp) {
      if (rec == cudaSuccess)
        rec = grp >= 2 ? launch_cols_batched(pj + jo, ps + so, pcount[grp], pblocks[grp], fmt, (grp & 1) ? 2 : 1,
                                             plan->cap, &launches)
                       : launch_pack_batched(pj + jo, ps + so, pcount[grp], pblocks[grp], fmt, (grp & 1) ? 2 : 1,
                                             plan->cap, &launches);
      jo += pcount[grp];
      so += pcount[grp] + 1;
    }
  }
  if (rec == cudaSuccess)
    rec = launch_tc_batched(fmt, reinterpret_cast<const TcJob*>(dbase + off_tjobs),
                            reinterpret_cast<const int*>(dbase + off_tilejob), nl, tiles, ctx->d_status,
                            ctx->wait_limit_ns, ctx->num_sms, plan->cap, &launches);
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
  err = cudaGraphLaunch(plan->exec, ctx->stream);
  if (err != cudaSuccess) {
    ctx->last_error = cudaGetErrorString(err);
    return M4RIE_ERR_CUDA;
  }
  ctx->launches += launches;
  return M4RIE_OK;
}

}  // namespace m4rie
