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
struct TrsmGraph;
void destroy_trsm_graph(TrsmGraph* g);
struct TuneEntry {
  int form = 0, sched = 0, group_m = 0;
  double ms = 0;
};
int shape_class(int64_t m, int64_t n, int64_t k);  // floor(log2(m*n*k)), tune.cu
// Operands of one product: A m x k, B k x n, C m x n, row strides in elements.
constexpr int kIoPanelsMax = 8;  // row panels of a pipelined host-buffer product, at most
constexpr size_t kPanelHostBytes = 1024;  // pinned pivot list of an echelon / PLE panel

struct Mats {
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  void* C;
  int64_t ldc;
};
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
  // tcgen05 GEMMs: 3 = 2-SM pairs (cta_group::2, default); 1 = single CTAs
  // (M4RIE_TC_CLUSTER)
  int cluster = 3;
  // kernels of a product launch with programmatic dependent launch, so each
  // one's launch and prologue overlap the previous one's tail (M4RIE_PDL=0: off)
  int pdl = 1;
  // Karatsuba on tcgen05 2-SM pairs (e <= 8) can recombine in the GEMM's
  // epilogue (M4RIE_FUSE_RECOMBINE=1).  Off by default: it runs every product
  // of an output tile back to back, and that tile order costs the GEMM more
  // L2 misses than the recombination kernel costs.
  int fuse_recombine = 0;
  // batched products: schedule per product (M4RIE_BATCHED_SCHED: alpha_b,
  // karatsuba, or auto: Karatsuba for e >= batched_kara_min_e and m n k >=
  // batched_kara_min_mnk, M4RIE_BATCHED_KARA_MIN_E / _MIN_MNK)
  int batched_sched = M4RIE_SCHED_AUTO;
  int batched_kara_min_e = 3;
  double batched_kara_min_mnk = 0;
  // m4rie_tune_batched: measured schedule and tile width (group_m: 1 wide,
  // 2 narrow) per [e][floor(log2(m n k))] (sched 0: not tuned);
  // batched_force(_width): what a tuning run imposes
  m4rie::TuneEntry btuned[11][64];
  int batched_force = 0, batched_force_width = 0;
  // m4rie_mul_host: kernels use pinned, device-mapped host buffers of small
  // products in place (M4RIE_ZERO_COPY=0: always staging copies)
  int zero_copy = 1;
  // pipelined host-buffer products: copy streams and their events
  cudaStream_t s_in = nullptr, s_out = nullptr;
  // echelon form and PLE look-ahead: side stream, its two events, pinned
  // pivot list of m4rie::kPanelHostBytes
  cudaStream_t ech_side = nullptr;
  cudaEvent_t ech_ev[2] = {};
  void* ech_po_host = nullptr;
  cudaEvent_t io_ev[2 * m4rie::kIoPanelsMax] = {};
  int io_panels = 4;  // row panels of a pipelined host-buffer product (M4RIE_IO_PANELS, 1..8)
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
  // triangular solves (trsm.cu): diagonal-block inverses, a row panel, the
  // log / antilog tables of the field last used
  void* tws = nullptr;
  size_t tws_bytes = 0;
  uint16_t* d_gf = nullptr;
  int gf_e = 0;
  uint32_t gf_f = 0;
  m4rie::TrsmGraph* trsm_graph = nullptr;  // the last solve, recorded for replay
  // echelon forms (echelon.cu): candidate lists, multipliers, panel products
  void* ews = nullptr;
  size_t ews_bytes = 0;
  int* ews_host = nullptr;  // pinned: two slots of row-move lists
};

namespace m4rie {
// batched.cu: many products in one persistent launch, replayed from a CUDA graph.
m4rie_status run_batched(m4rie_ctx* ctx, int count, const m4rie_problem* problems, int fmt);
// api.cu: one product with strided operands (validated, then dispatched by form and schedule).
// c_over_b (with add == 0): C may be B itself.  Every form reads B only while
// packing its operand planes, and the kernels that write C run after the
// packing kernels on the same stream, so C = A * B in place is safe.
m4rie_status run_gemm(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k, const Mats& x, int add,
                      bool c_over_b = false);
// run_gemm with the form and schedule given (>= 0) instead of resolved, and
// reuse_b: the B planes from the previous call on this B (same form,
// schedule, n, k) are reused.  The row panels of one host-buffer product.
m4rie_status run_gemm_as(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k, const Mats& x, int add,
                         bool c_over_b, int form_as, int sched_as, bool reuse_b);
}  // namespace m4rie

