// The context object behind m4rie_ctx (shared by api.cu and batched.cu).
#pragma once
#include <string>
#include <utility>
#include <vector>

#include "../../include/m4rie_gpu.h"
#include "m4rie_internal.cuh"

namespace m4rie {
struct BatchedPlan;
void destroy_plan(BatchedPlan* plan);
struct TuneEntry {
  int form = 0, sched = 0, group_m = 0;
  double ms = 0;
};
int shape_class(int64_t m, int64_t n, int64_t k);  // floor(log2(m*n*k)), tune.cu
}  // namespace m4rie

struct m4rie_ctx {
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* io = nullptr;  // device copies for m4rie_mul_host
  size_t io_bytes = 0;
  int* d_status = nullptr;
  int form = M4RIE_FORM_AUTO;
  int schedule = M4RIE_SCHED_AUTO;
  std::string last_error;
  int64_t launches = 0;
  uint64_t wait_limit_ns = 4000000000ull;
  int tc_chunk = 4096;  // elements of K' per FP32 accumulation chunk
  int f4nv = 0;         // FP4 form: kind::mxf4nvf4 instead of kind::mxf4
  int stall_test = 0;   // m4rie_set_test_hook flag 1
  int cluster = 2;      // tcgen05 GEMMs: 2-CTA clusters sharing B tiles (M4RIE_TC_CLUSTER=1: single CTAs)
  int group_m = 0;      // tcgen05 tile raster: m-tiles per column group (0: all m-tiles)
  m4rie::TuneEntry tuned[11][64];  // [e][floor(log2(m*n*k))] -> autotuned choice (form 0: none)
  // phase timing (m4rie_enable_timing)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;  // (phase, (start, stop))
  size_t ev_next = 0;
  double phase_ms[3] = {0, 0, 0};
  int64_t timed_products = 0;
  // cached plan + CUDA graph of the last batched call (batched.cu)
  m4rie::BatchedPlan* plan = nullptr;
};

namespace m4rie {
// batched.cu: many products in one persistent launch, replayed from a CUDA graph.
m4rie_status run_batched(m4rie_ctx* ctx, int count, const m4rie_problem* problems, int fmt);
}  // namespace m4rie

