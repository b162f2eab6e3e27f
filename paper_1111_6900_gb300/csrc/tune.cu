// Autotuner: picks the form, the schedule and the tile raster of the tcgen05
// GEMM for a shape class by measurement, and keeps the choices in the context
// (optionally in a text cache file).
//
// m4rie_tune runs every candidate on synthetic inputs of the requested shape
// (uniform field elements from a counter-based hash), checks that every
// candidate reproduces the first candidate's output bit for bit, times each
// one with CUDA events on the context's stream, and records the fastest for
// AUTO.  Shape classes are (e, floor(log2(m*n*k))).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "context.h"
#include "schedule.h"

namespace m4rie {
namespace {

// Field elements from a counter-based hash (splitmix64 finaliser) of the index.
__global__ void fill_elements(void* X, int64_t count, int eb, uint32_t emask, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    if (eb == 1) static_cast<uint8_t*>(X)[i] = (uint8_t)(z & emask);
    else static_cast<uint16_t*>(X)[i] = (uint16_t)(z & emask);
  }
}

__global__ void compare_bytes(const uint8_t* a, const uint8_t* b, int64_t n, int* diff) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (a[i] != b[i]) {
      atomicOr(diff, 1);
      return;
    }
}

}  // namespace

cudaError_t launch_fill_elements(void* X, int64_t count, int eb, uint32_t emask, uint64_t seed, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  fill_elements<<<(unsigned)std::min<int64_t>(ceil_div(count, 256), 4096), 256, 0, s>>>(X, count, eb, emask, seed);
  return cudaGetLastError();
}

int shape_class(int64_t m, int64_t n, int64_t k) {
  const double v = std::max(1.0, (double)m * (double)n * (double)k);
  return std::min(63, (int)std::floor(std::log2(v)));
}

}  // namespace m4rie

using namespace m4rie;

extern "C" {

m4rie_status m4rie_tune(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k) {
  if (!ctx) return M4RIE_ERR_ARG;
  m4rie_status st = m4rie_validate(e, f, m, n, k, (void*)16, (void*)32, (void*)48);
  if (st != M4RIE_OK && st != M4RIE_ERR_ALIAS) return st;
  if (m <= 0 || n <= 0 || k <= 0) return M4RIE_ERR_ARG;
  const int eb = e <= 8 ? 1 : 2;
  const size_t sa = (size_t)(m * k) * eb, sb = (size_t)(k * n) * eb, sc = (size_t)(m * n) * eb;
  uint8_t *A = nullptr, *B = nullptr, *C0 = nullptr, *C1 = nullptr;
  int* diff = nullptr;
  cudaError_t err = cudaMalloc(&A, sa);
  if (err == cudaSuccess) err = cudaMalloc(&B, sb);
  if (err == cudaSuccess) err = cudaMalloc(&C0, sc);
  if (err == cudaSuccess) err = cudaMalloc(&C1, sc);
  if (err == cudaSuccess) err = cudaMalloc(&diff, sizeof(int));
  auto cleanup = [&]() {
    cudaFree(A);
    cudaFree(B);
    cudaFree(C0);
    cudaFree(C1);
    cudaFree(diff);
  };
  if (err != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return M4RIE_ERR_NOMEM;
  }
  fill_elements<<<1024, 256, 0, ctx->stream>>>(A, m * k, eb, (1u << e) - 1, 0x1234ull);
  fill_elements<<<1024, 256, 0, ctx->stream>>>(B, k * n, eb, (1u << e) - 1, 0x5678ull);

  struct Cand {
    int form, sched, group_m;
  };
  std::vector<Cand> cands;
  for (int form : {M4RIE_FORM_POPC, M4RIE_FORM_TC_F8, M4RIE_FORM_TC_F4})
    for (int sched : {M4RIE_SCHED_ALPHA_B, M4RIE_SCHED_KARATSUBA}) {
      if (form == M4RIE_FORM_POPC) cands.push_back({form, sched, 0});
      else
        for (int gm : {0, 8}) cands.push_back({form, sched, gm});
    }
  cands.push_back({M4RIE_FORM_NEWTON_JOHN, M4RIE_SCHED_ALPHA_B, 0});  // no slicing: the schedule is unused
  const int saved_form = ctx->form, saved_sched = ctx->schedule, saved_gm = ctx->group_m;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  int best = -1;
  for (size_t c = 0; c < cands.size(); ++c) {
    ctx->form = cands[c].form;
    ctx->schedule = cands[c].sched;
    ctx->group_m = cands[c].group_m;
    uint8_t* out = c == 0 ? C0 : C1;
    st = m4rie_mul(ctx, e, f, m, n, k, A, B, out);  // warm-up and result
    if (st != M4RIE_OK) continue;
    if (c > 0) {
      cudaMemsetAsync(diff, 0, sizeof(int), ctx->stream);
      compare_bytes<<<1024, 256, 0, ctx->stream>>>(C0, C1, (int64_t)sc, diff);
      int h = 0;
      cudaMemcpyAsync(&h, diff, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
      cudaStreamSynchronize(ctx->stream);
      if (h) {
        ctx->last_error = "autotuner: a candidate disagreed with the reference result";
        continue;  // never pick a candidate that does not reproduce the product
      }
    }
    const int reps = 3;
    cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < reps; ++r) m4rie_mul(ctx, e, f, m, n, k, A, B, out);
    cudaEventRecord(e1, ctx->stream);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (ms < best_ms) {
      best_ms = ms;
      best = (int)c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->form = saved_form;
  ctx->schedule = saved_sched;
  ctx->group_m = saved_gm;
  err = cudaStreamSynchronize(ctx->stream);
  cleanup();
  if (err != cudaSuccess) {
    ctx->last_error = cudaGetErrorString(err);
    return M4RIE_ERR_CUDA;
  }
  if (best < 0) return M4RIE_ERR_CUDA;
  TuneEntry& t = ctx->tuned[e][shape_class(m, n, k)];
  t.form = cands[best].form;
  t.sched = cands[best].sched;
  t.group_m = cands[best].group_m;
  t.ms = best_ms;
  return M4RIE_OK;
}

m4rie_status m4rie_tuned_choice(m4rie_ctx* ctx, int e, int64_t m, int64_t n, int64_t k, int* form, int* schedule,
                                double* ms) {
  if (!ctx || e < 2 || e > 10) return M4RIE_ERR_ARG;
  const TuneEntry& t = ctx->tuned[e][shape_class(m, n, k)];
  if (form) *form = t.form;
  if (schedule) *schedule = t.sched;
  if (ms) *ms = t.ms;
  return M4RIE_OK;
}

m4rie_status m4rie_tune_save(m4rie_ctx* ctx, const char* path) {
  if (!ctx || !path) return M4RIE_ERR_ARG;
  FILE* fp = fopen(path, "w");
  if (!fp) return M4RIE_ERR_ARG;
  fprintf(fp, "# m4rie tune cache: e shape_class form schedule group_m ms\n");
  for (int e = 2; e <= 10; ++e)
    for (int c = 0; c < 64; ++c) {
      const TuneEntry& t = ctx->tuned[e][c];
      if (t.form) fprintf(fp, "%d %d %d %d %d %.6f\n", e, c, t.form, t.sched, t.group_m, t.ms);
    }
  // batched products (m4rie_tune_batched): "B e shape_class form schedule tile_width ms"
  for (int e = 2; e <= 10; ++e)
    for (int c = 0; c < 64; ++c) {
      const TuneEntry& t = ctx->btuned[e][c];
      if (t.sched) fprintf(fp, "B %d %d %d %d %d %.6f\n", e, c, t.form, t.sched, t.group_m, t.ms);
    }
  fclose(fp);
  return M4RIE_OK;
}

m4rie_status m4rie_tune_load(m4rie_ctx* ctx, const char* path) {
  if (!ctx || !path) return M4RIE_ERR_ARG;
  FILE* fp = fopen(path, "r");
  if (!fp) return M4RIE_ERR_ARG;
  char line[256];
  while (fgets(line, sizeof(line), fp)) {
    if (line[0] == '#') continue;
    int e, c, form, sched, gm;
    double ms;
    if (line[0] == 'B') {
      int width = 0;
      if (sscanf(line + 1, "%d %d %d %d %d %lf", &e, &c, &form, &sched, &width, &ms) == 6 && e >= 2 && e <= 10 &&
          c >= 0 && c < 64 && (form == M4RIE_FORM_TC_F4 || form == M4RIE_FORM_TC_F8) &&
          sched >= M4RIE_SCHED_ALPHA_B && sched <= M4RIE_SCHED_KARATSUBA && width >= 0 && width <= 2)
        ctx->btuned[e][c] = TuneEntry{form, sched, width, ms};
      continue;
    }
    if (sscanf(line, "%d %d %d %d %d %lf", &e, &c, &form, &sched, &gm, &ms) != 6) continue;
    if (e < 2 || e > 10 || c < 0 || c > 63 || form < M4RIE_FORM_POPC || form > M4RIE_FORM_NEWTON_JOHN ||
        sched < M4RIE_SCHED_ALPHA_B || sched > M4RIE_SCHED_KARATSUBA || gm < 0)
      continue;
    ctx->tuned[e][c] = TuneEntry{form, sched, gm, ms};
  }
  fclose(fp);
  return M4RIE_OK;
}

}  // extern "C"
