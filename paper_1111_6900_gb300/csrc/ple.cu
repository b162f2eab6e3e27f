// PLE decomposition over GF(2^e) (Section 4.2): A = P L E in place, in the
// library's variant of the definition (E has leading 1s, L holds the pivots
// on its diagonal), with Algorithm 4's pivoting: for every column the first
// row at or below the current rank with a non-zero entry is swapped up.
//
// Layout of the result (rank r): A[i][t] = L[i][t] for t <= min(i, r - 1);
// for k < r, E[k][j] = A[k][j] for j > Q[k] (E[k][Q[k]] = 1 is not stored);
// every other entry is 0.  P[t] is the row swapped with row t at step t and
// Q[t] the pivot column of step t.  This is the matrix that Algorithm 4 with
// Section 4.2's changes leaves (the multipliers kept in place as L, the rows
// above the pivot untouched), once L's columns are moved next to the
// diagonal.  Here they are written there directly: L's column t goes to
// column t as soon as pivot t is known.
//
// The elimination runs by panels of W = 64 columns; a panel takes one or
// more rounds:
//
//   1. Panel kernel (one CTA, bit slices in registers, Section 3.2): the
//      candidates are the next R = 96 rows at or below the rank, in their
//      current order.  Column by column, the candidate at the lowest current
//      position with a non-zero entry is the pivot; it takes the position of
//      the next pivot and the row there takes its old one (Algorithm 4's
//      swap); the candidates that are not yet pivots get the multiple of the
//      pivot row that clears the column.  The round stops at the first column
//      where no candidate has a non-zero entry (column j0), unless the
//      candidates are all the remaining rows: then that column has no pivot
//      and the round goes on.  Out: the pivots
//      and their swaps, E's rows over the panel (the pivot rows scaled to a
//      leading 1), Lp^{-1} (Lp: L's block of the round's pivot rows; the
//      kernel tracks each pivot row's combination of the original rows), and
//      the pivot rows' final entries in the panel and in L's columns.
//   2. The host replays the round's swaps on the candidate block (one move of
//      whole rows).
//   3. Apply kernel (two threads per row, one per 32-column word): every
//      other remaining row is eliminated with E's rows over the panel, its
//      multipliers are written to L's columns r .. r+k-1, and the first row
//      with a non-zero entry in column j0 is found.
//   4. Right of the panel: G = Lp^{-1} (pivot rows) is E's rows there (one
//      product, copied into the pivot rows), and the remaining rows get
//      L G added (one product).
//   5. With j0 inside the panel: the row found in 3 is swapped up (the pivot
//      of column j0) and another round starts at column j0; with none, column
//      j0 has no pivot and the next round starts after it.
//
// Random dense input finds all 64 pivots of a panel in one round.  After a
// panel's last round, the next panel's kernel starts on a side stream as
// soon as L and G are known: it gives its own candidate block (96 rows x 64
// columns) the update L G itself, and the products of step 4 skip that
// block, so they run beside it.
#include <algorithm>
#include <climits>
#include <numeric>
#include <vector>

#include "context.h"
#include "bitslice.cuh"
#include "rowmove.cuh"

namespace m4rie {

// trsm.cu: log / antilog tables of the field in the context: log at
// [0, 1024) (log 0 = 2(2^e - 1)), antilog at [1024, 5120).
m4rie_status ensure_field_tables(m4rie_ctx* ctx, int e, uint32_t f);

namespace {

using namespace bitslice;

constexpr int W = 64;                // panel columns
constexpr int R = rowmove::kRows;    // candidate rows per round
constexpr int LOGW = 1024;           // log table entries
constexpr int EXPW = 4096;           // antilog entries (doubled, then zeros)
constexpr int PT = 4 * R;            // panel kernel threads: (row, word) for 96 rows x 4 words
constexpr int AT = 64;               // apply kernel threads: 32 rows x 2 words
constexpr int ESL_MAX = W * 10 * 2;  // E's rows as slices: [pivot][slice][word]
// Largest e for which the next panel's kernel applies the previous panel's
// update to its candidate block itself (its cost grows as e^2 per step).
constexpr int kPreUpdateMaxE = 4;

struct PleOut {
  int k;        // pivots of the round
  int j0;       // panel column where the round stopped (wc: at the panel's end)
  int pos[W];   // window position of pivot a's row before its swap
  int cols[W];  // panel column of pivot a
};
static_assert(sizeof(PleOut) <= kPanelHostBytes, "pinned pivot list");

// Step 1 on the candidate block A[r .. r+cnt) over panel columns [js, wc)
// (columns left of js are closed: they hold L entries or zeros).  Thread
// (row, word): words 0 and 1 are the row's panel columns as E slices, words
// 2 and 3 its combination of the original candidate rows, indexed by pivot
// number (a pivot row has coefficient 1 at its own number).  Only rows that
// are not pivots are eliminated, so pivot row a ends as pv_a E_a with the
// combination pv_a (Lp^{-1} row a): Lp^{-1}[a][b] = pv_a^{-1} times the
// combination's entry b.  lrec keeps every candidate's multiplier at every
// step it is eliminated in (L's entries of the later pivot rows).
//
// With kp > 0 the candidate block first gets the previous panel's update:
// block += pl[row][0 .. kp) times px's first wc columns (pl: the previous
// panel's multipliers of these rows, stride W; px: its G, row stride ldx),
// which is then written back to A (the update of the rest of the matrix
// skips this block).
//
// One barrier per column: before it, every thread stores its slices (a
// snapshot, two buffers used alternately) and each warp offers its best
// candidate, (position, row, entry) packed so that the minimum is the
// candidate at the lowest current position; after it, the pivot's slices
// are read from the snapshot.  The pivot's own coefficient bit is not in
// the snapshot; the rows it eliminates add it themselves.  Positions live in
// registers: the pivot takes position k, the row at position k the pivot's
// old one (Algorithm 4's swap).
template <typename T, int E>
__global__ void __launch_bounds__(PT) ple_panel(T* __restrict__ A, int64_t lda, int64_t r, int64_t c0, int cnt,
                                                int wc, int js, uint32_t flow, const uint16_t* __restrict__ gf,
                                                PleOut* __restrict__ out, T* __restrict__ linv,
                                                uint32_t* __restrict__ esl, int* status, const T* __restrict__ pl,
                                                const T* __restrict__ px, int64_t ldx, int kp, int64_t m) {
  extern __shared__ uint32_t snap[];  // [2][E][PT], then the previous G's slices [W][E][2]
  uint32_t* xs = snap + 2 * E * PT;
  __shared__ uint16_t lg[LOGW];
  __shared__ uint16_t ex[EXPW];
  __shared__ unsigned cand[3];      // a column's pivot key (three, used in turn)
  __shared__ int piv_col[W], piv_pos[W];
  __shared__ uint32_t piv_val[W];
  __shared__ __align__(16) T lrec[R][W];
  const uint32_t q = (1u << E) - 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = warp * 8 + (lane >> 2), word = lane & 3;
  for (int i = tid; i < (int)(3 * q); i += PT) {
    if (i < (int)q) lg[i + 1] = gf[i + 1];
    else ex[i - q] = gf[LOGW + i - q];
  }
  if (tid < 3) cand[tid] = ~0u;
  uint32_t sl[E];
  bool bad = false;
  if (word < 2 && row < cnt) {
    bad = load_word<T, E>(A + (r + row) * lda + c0 + 32 * word, 32 * word, js, wc, sl);
  } else {
#pragma unroll
    for (int t = 0; t < E; ++t) sl[t] = 0;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kStatusRange);
  if (kp > 0) {
    // the previous panel's update of this block: its multipliers to lrec
    // (overwritten later, each entry before it is read), its G as slices
    constexpr int VPR = W * (int)sizeof(T) / 16;  // 16-byte vectors per row of pl and lrec
    const uint4* src4 = reinterpret_cast<const uint4*>(pl);
    uint4* dst4 = reinterpret_cast<uint4*>(&lrec[0][0]);
    for (int i = tid; i < cnt * VPR; i += PT) dst4[i] = src4[i];
    if (tid < 2 * kp) {
      uint32_t gs[E];
      load_word<T, E>(px + (int64_t)(tid >> 1) * ldx + 32 * (tid & 1), 32 * (tid & 1), 0, wc, gs);
#pragma unroll
      for (int t = 0; t < E; ++t) xs[((tid >> 1) * E + t) * 2 + (tid & 1)] = gs[t];
    }
    __syncthreads();
    if (word < 2 && row < cnt) {
      for (int a = 0; a < kp; ++a) {
        const uint32_t sa = lrec[row][a];
        if (sa) add_scaled<E>(sl, sa, &xs[a * E * 2 + word], 2, flow);
      }
      T* dst = A + (r + row) * lda + c0 + 32 * word;
      for (int b = 0; b < 32 && 32 * word + b < wc; ++b) dst[b] = (T)element_at<E>(sl, b);
    }
  }
  __syncthreads();

  // Rows at or past cnt hold zeros: they never offer a pivot and are never
  // eliminated.
  int k = 0, my_a = -1, j0 = wc;
  int slot = 0;      // cand slot of this column (0, 1, 2 in turn)
  int sbuf = 0;      // snapshot buffer of this column (0 or E PT, alternately)
  int mypos = row;   // current window position of this row
  for (int j = js; j < wc; ++j) {
    const int wj = j >> 5, bj = j & 31;
    uint32_t x = word == wj ? element_at<E>(sl, bj) : 0u;
    x = __shfl_sync(0xffffffffu, x, (lane & ~3) | wj);  // the entry at column j, to the row's four lanes
    const uint32_t lx = x ? lg[x] : 0u;                  // its logarithm, looked up before the barrier
    uint32_t* sn = snap + sbuf;
#pragma unroll
    for (int t = 0; t < E; ++t) sn[t * PT + tid] = sl[t];
    const bool hit = word == wj && my_a < 0 && x != 0;
    const unsigned key = hit ? ((unsigned)mypos << 17) | ((unsigned)row << 10) | lx : ~0u;
    const unsigned wmin = __reduce_min_sync(0xffffffffu, key);
    if (lane == 0 && wmin != ~0u) atomicMin(&cand[slot], wmin);
    __syncthreads();
    const unsigned c = cand[slot];
    // the slot of the column after next: its last reads were before this
    // barrier, its next writes come after the next one
    if (tid == 0) cand[slot == 0 ? 2 : slot - 1] = ~0u;
    slot = slot == 2 ? 0 : slot + 1;
    sbuf = sbuf ? 0 : E * PT;
    if (c == ~0u) {  // no candidate has a non-zero entry here (uniform)
      // with every remaining row a candidate, no row has one: no pivot here
      if (cnt == m - r) continue;
      j0 = j;  // a row below the candidates may have one: the round ends
      break;
    }
    const int p = (int)((c >> 10) & 127u), old = (int)(c >> 17);
    const uint32_t lpv = c & 1023u;  // log of the pivot
    if (row == p) {
      my_a = k;
      mypos = k;
      if (word == 2 + (k >> 5)) sl[0] ^= 1u << (k & 31);  // coefficient 1 on its own original row
      if (word == 0) {
        piv_col[k] = j;
        piv_val[k] = x;
        piv_pos[k] = old;
      }
    } else {
      if (mypos == k) mypos = old;
      if (my_a < 0 && word == 0) lrec[row][k] = (T)x;
    }
    if (my_a < 0 && x != 0) {
      // row += (x / pv) * pivot row, slice by slice, and the pivot's own bit
      const uint32_t s2 = ex[lx + q - lpv];
      add_scaled<E>(sl, s2, &sn[p * 4 + word], PT, flow);
      if (word == 2 + (k >> 5)) {
#pragma unroll
        for (int t = 0; t < E; ++t) sl[t] ^= ((s2 >> t) & 1u) << (k & 31);
      }
    }
    ++k;
  }

  if (my_a >= 0) {
    const uint32_t pv = piv_val[my_a];
    const uint32_t lpv = lg[pv];
    T* dst = A + (r + row) * lda;
    if (word < 2) {
      // E's row: the pivot row scaled by pv^{-1}
      uint32_t es[E];
      scaled<E>(es, ex[q - lpv], sl, flow);
#pragma unroll
      for (int t = 0; t < E; ++t) esl[(my_a * E + t) * 2 + word] = es[t];
      // its entries right of L's columns: 0 up to the pivot column, then E
      const int qa = piv_col[my_a];
      for (int b = 0; b < 32; ++b) {
        const int cc = 32 * word + b;
        if (cc >= wc) break;
        if (cc < js || c0 + cc <= r + my_a) continue;
        dst[c0 + cc] = (T)(cc <= qa ? 0u : element_at<E>(es, b));
      }
    } else {
      const int b0 = 32 * (word - 2);
      // L's entries of the row: the multipliers, then the pivot on the diagonal
      for (int s = b0; s < b0 + 32 && s <= my_a; ++s) dst[r + s] = s < my_a ? lrec[row][s] : (T)pv;
      // Lp^{-1}: the combination scaled by pv^{-1}
      for (int bb = 0; bb < 32; ++bb) {
        const int b = b0 + bb;
        if (b >= k) break;
        const uint32_t v = element_at<E>(sl, bb);
        linv[my_a * W + b] = (T)(v ? ex[lg[v] + q - lpv] : 0u);
      }
    }
  }
  if (tid == 0) {
    out->k = k;
    out->j0 = j0;
  }
  for (int a = tid; a < k; a += PT) {
    out->pos[a] = piv_pos[a];
    out->cols[a] = piv_col[a];
  }
}

// Step 3 on rows [i_begin, m): each row is eliminated with E's rows over the
// open panel columns [js, wc) in pivot order (E_a has a 1 in column cols[a],
// so the multiplier is the row's entry there at step a, which becomes
// L[i][r + a]).  Written back: L's entries to columns r .. r+k-1 of A and to
// lbuf (row i - i_begin, stride W), the panel columns right of them.  With
// j0 < wc, the lowest row with a non-zero entry in column j0 goes to *first.
template <typename T, int E>
__global__ void __launch_bounds__(AT) ple_apply(T* __restrict__ A, int64_t lda, int64_t i_begin, int64_t m,
                                                int64_t r, int64_t c0, int wc, int js, int k, int j0,
                                                uint32_t flow, const PleOut* __restrict__ po,
                                                const uint32_t* __restrict__ esl, T* __restrict__ lbuf,
                                                int* __restrict__ first, int* status) {
  __shared__ uint32_t es[ESL_MAX];
  __shared__ int qc[W];
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < k * E * 2; i += AT) es[i] = esl[i];
  for (int i = tid; i < k; i += AT) qc[i] = po->cols[i];
  __syncthreads();
  const int64_t i = i_begin + (int64_t)blockIdx.x * (AT / 2) + (tid >> 1);
  const int word = tid & 1;
  const bool live = i < m;
  uint32_t sl[E], ls[E];
#pragma unroll
  for (int t = 0; t < E; ++t) sl[t] = ls[t] = 0;
  bool bad = false;
  T* rowp = A + (live ? i : i_begin) * lda;
  if (live) bad = load_word<T, E>(rowp + c0 + 32 * word, 32 * word, js, wc, sl);
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kStatusRange);
  for (int a = 0; a < k; ++a) {
    const int qa = qc[a], wq = qa >> 5;
    uint32_t x = word == wq ? element_at<E>(sl, qa & 31) : 0u;
    x = __shfl_sync(0xffffffffu, x, (lane & ~1) | wq);
    if (word == (a >> 5)) {
#pragma unroll
      for (int t = 0; t < E; ++t) ls[t] |= ((x >> t) & 1u) << (a & 31);
    }
    if (x) add_scaled<E>(sl, x, &es[a * E * 2 + word], 2, flow);
  }
  if (!live) return;
  if (k > 0) {
    const int b0 = 32 * word;
    T* lrow = lbuf + (i - i_begin) * W;
    for (int s = b0; s < b0 + 32 && s < k; ++s) {
      const T v = (T)element_at<E>(ls, s - b0);
      rowp[r + s] = v;
      lrow[s] = v;
    }
    for (int b = 0; b < 32; ++b) {
      const int c = b0 + b;
      if (c >= wc) break;
      if (c < js || c0 + c < r + k) continue;
      rowp[c0 + c] = (T)element_at<E>(sl, b);
    }
  }
  if (j0 < wc && word == (j0 >> 5) && element_at<E>(sl, j0 & 31) != 0) atomicMin(first, (int)i);
}

// The previous panel's update of the candidate block (kp = 0: none).
// m: the matrix's rows (the panel kernel needs them to know whether its
// candidates are all the remaining rows).
template <typename T>
struct PreUpdate {
  const T* pl = nullptr;
  const T* px = nullptr;
  int64_t ldx = 0;
  int kp = 0;
  int64_t m = 0;
};

template <typename T, int E>
cudaError_t launch_panel_e(T* A, int64_t lda, int64_t r, int64_t c0, int cnt, int wc, int js, uint32_t flow,
                           const uint16_t* gf, PleOut* out, T* linv, uint32_t* esl, int* status,
                           const PreUpdate<T>& pre, cudaStream_t s) {
  // the two snapshots, then the previous G's slices
  constexpr int smem = (2 * E * PT + W * E * 2) * (int)sizeof(uint32_t);
  const cudaError_t err = cudaFuncSetAttribute(ple_panel<T, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (err != cudaSuccess) return err;
  ple_panel<T, E><<<1, PT, smem, s>>>(A, lda, r, c0, cnt, wc, js, flow, gf, out, linv, esl, status, pre.pl, pre.px,
                                      pre.ldx, pre.kp, pre.m);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_panel(int e, T* A, int64_t lda, int64_t r, int64_t c0, int cnt, int wc, int js, uint32_t f,
                         const uint16_t* gf, PleOut* out, T* linv, uint32_t* esl, int* status, cudaStream_t s,
                         const PreUpdate<T>& pre) {
  const uint32_t flow = f & ((1u << e) - 1u);
#define M4RIE_PLE_CASE(EE) \
  case EE:                 \
    return launch_panel_e<T, EE>(A, lda, r, c0, cnt, wc, js, flow, gf, out, linv, esl, status, pre, s);
  switch (e) {
    M4RIE_PLE_CASE(2)
    M4RIE_PLE_CASE(3)
    M4RIE_PLE_CASE(4)
    M4RIE_PLE_CASE(5)
    M4RIE_PLE_CASE(6)
    M4RIE_PLE_CASE(7)
    M4RIE_PLE_CASE(8)
    M4RIE_PLE_CASE(9)
    M4RIE_PLE_CASE(10)
    default: return cudaErrorInvalidValue;
  }
#undef M4RIE_PLE_CASE
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply(int e, T* A, int64_t lda, int64_t i_begin, int64_t m, int64_t r, int64_t c0, int wc, int js,
                         int k, int j0, uint32_t f, const PleOut* po, const uint32_t* esl, T* lbuf, int* first,
                         int* status, cudaStream_t s) {
  const uint32_t flow = f & ((1u << e) - 1u);
  const unsigned grid = (unsigned)ceil_div(m - i_begin, AT / 2);
#define M4RIE_PLE_CASE(EE)                                                                                       \
  case EE:                                                                                                       \
    ple_apply<T, EE><<<grid, AT, 0, s>>>(A, lda, i_begin, m, r, c0, wc, js, k, j0, flow, po, esl, lbuf, first, \
                                         status);                                                                \
    break;
  switch (e) {
    M4RIE_PLE_CASE(2)
    M4RIE_PLE_CASE(3)
    M4RIE_PLE_CASE(4)
    M4RIE_PLE_CASE(5)
    M4RIE_PLE_CASE(6)
    M4RIE_PLE_CASE(7)
    M4RIE_PLE_CASE(8)
    M4RIE_PLE_CASE(9)
    M4RIE_PLE_CASE(10)
    default: return cudaErrorInvalidValue;
  }
#undef M4RIE_PLE_CASE
  return cudaGetLastError();
}

using rowmove::fail;
using rowmove::move_rows;

// The context's products on another stream for the lifetime of the object.
struct OnStream {
  m4rie_ctx* ctx;
  cudaStream_t saved;
  OnStream(m4rie_ctx* c, cudaStream_t s) : ctx(c), saved(c->stream) { c->stream = s; }
  ~OnStream() { ctx->stream = saved; }
};

template <typename T>
m4rie_status ple_impl(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, T* A, int64_t lda, int64_t* rank,
                      int64_t* P, int64_t* Q) {
  const size_t w = sizeof(T);
  // workspace: pivot list and the row found in step 3; move lists; Lp^{-1};
  // E's slices; the multipliers of the remaining rows; G; the row-move scratch
  const size_t sz_small = round_up((int64_t)(sizeof(PleOut) + 64 + sizeof(int) * 2 * rowmove::kSlot), 256);
  const size_t sz_linv = round_up((int64_t)((size_t)W * W * w), 256);
  const size_t sz_esl = round_up((int64_t)(sizeof(uint32_t) * ESL_MAX), 256);
  const size_t sz_lbuf = round_up((int64_t)((size_t)m * W * w), 256);
  const size_t sz_X = round_up((int64_t)((size_t)W * n * w), 256);
  const size_t sz_tmp = round_up((int64_t)((size_t)2 * R * n * w), 256);
  const size_t total = sz_small + sz_linv + sz_esl + sz_lbuf + sz_X + sz_tmp;
  cudaError_t err;
  if (total > ctx->ews_bytes) {
    if ((err = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return fail(ctx, err);
    if (ctx->ews) cudaFree(ctx->ews);
    ctx->ews = nullptr;
    ctx->ews_bytes = 0;
    if (cudaMalloc(&ctx->ews, total) != cudaSuccess) {
      cudaGetLastError();
      ctx->last_error = "PLE workspace allocation failed";
      return M4RIE_ERR_NOMEM;
    }
    ctx->ews_bytes = total;
  }
  if (!ctx->ews_host && cudaMallocHost(&ctx->ews_host, sizeof(int) * 2 * rowmove::kSlot) != cudaSuccess) {
    cudaGetLastError();
    ctx->ews_host = nullptr;
    ctx->last_error = "pinned host buffer allocation failed";
    return M4RIE_ERR_NOMEM;
  }
  if ((err = rowmove::ensure_side(ctx)) != cudaSuccess) return fail(ctx, err);
  uint8_t* base = static_cast<uint8_t*>(ctx->ews);
  PleOut* d_po = reinterpret_cast<PleOut*>(base);
  int* d_first = reinterpret_cast<int*>(base + sizeof(PleOut));
  rowmove::Bufs mv;
  mv.moves = reinterpret_cast<int*>(base + sizeof(PleOut) + 64);
  mv.host = ctx->ews_host;
  T* linv = reinterpret_cast<T*>(base + sz_small);
  uint32_t* esl = reinterpret_cast<uint32_t*>(base + sz_small + sz_linv);
  T* lbuf = reinterpret_cast<T*>(base + sz_small + sz_linv + sz_esl);
  T* X = reinterpret_cast<T*>(base + sz_small + sz_linv + sz_esl + sz_lbuf);
  mv.tmp = base + sz_small + sz_linv + sz_esl + sz_lbuf + sz_X;
  PleOut* hpo_next = static_cast<PleOut*>(ctx->ech_po_host);
  PreUpdate<T> plain;  // no previous update to apply
  plain.m = m;

  std::vector<int64_t> piv(std::min(m, n)), perm(std::min(m, n));
  std::vector<int> src, dst, win;
  PleOut hpo;
  bool ahead = false;  // this panel's first kernel was launched by the previous panel
  int64_t r = 0;
  for (int64_t c0 = 0; c0 < n && r < m; c0 += W) {
    const int wc = (int)std::min<int64_t>(W, n - c0);
    const int64_t cr = c0 + wc, nb = n - cr;
    int js = 0;
    int64_t preswap = -1;  // the row swapped to position r for column js, if any
    while (js < wc && r < m) {
      const int cnt = (int)std::min<int64_t>(R, m - r);
      // 1. pivots of the candidate block
      if (js == 0 && ahead) {
        if ((err = cudaEventSynchronize(ctx->ech_ev[1])) != cudaSuccess ||
            (err = cudaStreamWaitEvent(ctx->stream, ctx->ech_ev[1], 0)) != cudaSuccess)
          return fail(ctx, err);
        hpo = *hpo_next;
        ahead = false;
      } else {
        if ((err = launch_panel<T>(e, A, lda, r, c0, cnt, wc, js, f, ctx->d_gf, d_po, linv, esl, ctx->d_status,
                                   ctx->stream, plain)) != cudaSuccess)
          return fail(ctx, err);
        ++ctx->launches;
        if ((err = cudaMemcpyAsync(&hpo, d_po, sizeof(PleOut), cudaMemcpyDeviceToHost, ctx->stream)) !=
                cudaSuccess ||
            (err = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
          return fail(ctx, err);
      }
      const int k = hpo.k, j0 = hpo.j0;
      if (k < 0 || k > std::min(cnt, wc - js) || j0 < js || j0 > wc || (preswap >= 0 && (k == 0 || hpo.pos[0] != 0))) {
        ctx->last_error = "PLE panel kernel returned an inconsistent pivot list";
        return M4RIE_ERR_CUDA;
      }
      // 2. the round's swaps on the candidate block, as moves of whole rows
      if (k > 0) {
        win.resize(cnt);
        std::iota(win.begin(), win.end(), 0);
        for (int a = 0; a < k; ++a) {
          const int pa = hpo.pos[a];
          if (pa < a || pa >= cnt) {
            ctx->last_error = "PLE panel kernel returned an inconsistent swap";
            return M4RIE_ERR_CUDA;
          }
          std::swap(win[a], win[pa]);
          perm[r + a] = (a == 0 && preswap >= 0) ? preswap : r + pa;
          piv[r + a] = c0 + hpo.cols[a];
        }
        src.clear();
        dst.clear();
        for (int x = 0; x < cnt; ++x)
          if (win[x] != x) {
            src.push_back((int)(r + win[x]));
            dst.push_back((int)(r + x));
          }
        if ((err = move_rows<T>(ctx, mv, 1, A, lda, 0, n, src, dst)) != cudaSuccess) return fail(ctx, err);
      }
      preswap = -1;
      // 3. G = Lp^{-1} (pivot rows) right of the panel, on the side stream,
      // beside the apply kernel on the other remaining rows (which also
      // finds the pivot row of column j0)
      const int64_t rest = m - (r + k);
      const bool open = j0 < wc;
      T* Ar = A + r * lda + cr;
      const bool right = k > 0 && nb > 0;
      if (right) {
        if ((err = cudaEventRecord(ctx->ech_ev[0], ctx->stream)) != cudaSuccess ||
            (err = cudaStreamWaitEvent(ctx->ech_side, ctx->ech_ev[0], 0)) != cudaSuccess)
          return fail(ctx, err);
        {
          OnStream on(ctx, ctx->ech_side);
          m4rie_status st = run_gemm(ctx, e, f, k, nb, k, Mats{linv, W, Ar, lda, X, nb}, 0);
          if (st != M4RIE_OK) return st;
        }
        if ((err = cudaEventRecord(ctx->ech_ev[1], ctx->ech_side)) != cudaSuccess) return fail(ctx, err);
      }
      if (rest > 0 && (k > 0 || open)) {
        if (open && (err = cudaMemsetAsync(d_first, 0x7f, sizeof(int), ctx->stream)) != cudaSuccess)
          return fail(ctx, err);
        if ((err = launch_apply<T>(e, A, lda, r + k, m, r, c0, wc, js, k, open ? j0 : wc, f, d_po, esl, lbuf,
                                   d_first, ctx->d_status, ctx->stream)) != cudaSuccess)
          return fail(ctx, err);
        ++ctx->launches;
      }
      // 4. the other remaining rows right of the panel get L G
      if (right) {
        if ((err = cudaStreamWaitEvent(ctx->stream, ctx->ech_ev[1], 0)) != cudaSuccess) return fail(ctx, err);
        m4rie_status st;
        if (rest > 0) {
          const int64_t r_next = r + k;
          T* Ad = A + r_next * lda + cr;
          const bool look = !open && nb > 2 * W;
          if (look && e <= kPreUpdateMaxE) {
            // Look-ahead: the next panel's kernel gives its own candidate
            // block (rows r_next.., the next W columns) this update and
            // starts now, beside the update of the rest of the matrix.
            const int cnt_next = (int)std::min<int64_t>(R, rest);
            PreUpdate<T> pre;
            pre.pl = lbuf;
            pre.px = X;
            pre.ldx = nb;
            pre.kp = k;
            pre.m = m;
            if ((err = cudaEventRecord(ctx->ech_ev[0], ctx->stream)) != cudaSuccess ||
                (err = cudaStreamWaitEvent(ctx->ech_side, ctx->ech_ev[0], 0)) != cudaSuccess ||
                (err = launch_panel<T>(e, A, lda, r_next, cr, cnt_next, W, 0, f, ctx->d_gf, d_po, linv, esl,
                                       ctx->d_status, ctx->ech_side, pre)) != cudaSuccess ||
                (err = cudaMemcpyAsync(hpo_next, d_po, sizeof(PleOut), cudaMemcpyDeviceToHost, ctx->ech_side)) !=
                    cudaSuccess ||
                (err = cudaEventRecord(ctx->ech_ev[1], ctx->ech_side)) != cudaSuccess)
              return fail(ctx, err);
            ++ctx->launches;
            ahead = true;
            // the candidate rows right of that block, then every row below them
            if ((st = run_gemm(ctx, e, f, cnt_next, nb - W, k, Mats{lbuf, W, X + W, nb, Ad + W, lda}, 1)) !=
                M4RIE_OK)
              return st;
            if (rest > cnt_next &&
                (st = run_gemm(ctx, e, f, rest - cnt_next, nb, k,
                               Mats{lbuf + (int64_t)cnt_next * W, W, X, nb, Ad + (int64_t)cnt_next * lda, lda}, 1)) !=
                    M4RIE_OK)
              return st;
          } else if (look) {
            // Look-ahead for larger fields, where the block's update costs the
            // one-CTA kernel more than a product: the next panel's columns
            // first, then its kernel beside the rest of the update.
            const int cnt_next = (int)std::min<int64_t>(R, rest);
            if ((st = run_gemm(ctx, e, f, rest, W, k, Mats{lbuf, W, X, nb, Ad, lda}, 1)) != M4RIE_OK) return st;
            if ((err = cudaEventRecord(ctx->ech_ev[0], ctx->stream)) != cudaSuccess ||
                (err = cudaStreamWaitEvent(ctx->ech_side, ctx->ech_ev[0], 0)) != cudaSuccess ||
                (err = launch_panel<T>(e, A, lda, r_next, cr, cnt_next, W, 0, f, ctx->d_gf, d_po, linv, esl,
                                       ctx->d_status, ctx->ech_side, plain)) != cudaSuccess ||
                (err = cudaMemcpyAsync(hpo_next, d_po, sizeof(PleOut), cudaMemcpyDeviceToHost, ctx->ech_side)) !=
                    cudaSuccess ||
                (err = cudaEventRecord(ctx->ech_ev[1], ctx->ech_side)) != cudaSuccess)
              return fail(ctx, err);
            ++ctx->launches;
            ahead = true;
            if ((st = run_gemm(ctx, e, f, rest, nb - W, k, Mats{lbuf, W, X + W, nb, Ad + W, lda}, 1)) != M4RIE_OK)
              return st;
          } else if ((st = run_gemm(ctx, e, f, rest, nb, k, Mats{lbuf, W, X, nb, Ad, lda}, 1)) != M4RIE_OK) {
            return st;
          }
        }
        if ((err = cudaMemcpy2DAsync(Ar, (size_t)lda * w, X, (size_t)nb * w, (size_t)nb * w, (size_t)k,
                                     cudaMemcpyDeviceToDevice, ctx->stream)) != cudaSuccess)
          return fail(ctx, err);
      }
      r += k;
      if (!open) break;
      // 5. column j0: its pivot row, found in step 3, swapped up; or no pivot
      int first = INT_MAX;
      if (rest > 0) {
        if ((err = cudaMemcpyAsync(&first, d_first, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream)) !=
                cudaSuccess ||
            (err = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
          return fail(ctx, err);
      }
      if (first != 0x7f7f7f7f && first != INT_MAX) {
        if (first < r || first >= m) {
          ctx->last_error = "PLE apply kernel returned an inconsistent row";
          return M4RIE_ERR_CUDA;
        }
        if (first != r) {
          src.assign({(int)r, first});
          dst.assign({first, (int)r});
          if ((err = move_rows<T>(ctx, mv, 0, A, lda, 0, n, src, dst)) != cudaSuccess) return fail(ctx, err);
        }
        preswap = first;
        js = j0;
      } else {
        js = j0 + 1;
      }
    }
  }
  if (ahead && (err = cudaEventSynchronize(ctx->ech_ev[1])) != cudaSuccess) return fail(ctx, err);
  if ((err = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return fail(ctx, err);
  if (rank) *rank = r;
  if (P) {
    for (int64_t i = 0; i < m; ++i) P[i] = i;
    for (int64_t i = 0; i < r; ++i) P[i] = perm[i];
  }
  if (Q) {
    for (int64_t j = 0; j < n; ++j) Q[j] = j;
    for (int64_t i = 0; i < r; ++i) Q[i] = piv[i];
  }
  return M4RIE_OK;
}

}  // namespace
}  // namespace m4rie

using namespace m4rie;

extern "C" {

m4rie_status m4rie_ple(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, void* A, int64_t lda, int64_t* rank,
                       int64_t* P, int64_t* Q) {
  if (!ctx) return M4RIE_ERR_ARG;
  m4rie_status st = m4rie_validate(e, f, 0, 0, 0, nullptr, nullptr, nullptr);
  if (st != M4RIE_OK) return st;
  if (m < 0 || n < 0 || m > (1ll << 31) - 1 || n > (1ll << 31) - 1 || lda < n || (m > 0 && n > 0 && !A))
    return M4RIE_ERR_ARG;
  if (rank) *rank = 0;
  if (P)
    for (int64_t i = 0; i < m; ++i) P[i] = i;
  if (Q)
    for (int64_t j = 0; j < n; ++j) Q[j] = j;
  if (m == 0 || n == 0) return M4RIE_OK;
  if ((st = ensure_field_tables(ctx, e, f)) != M4RIE_OK) return st;
  if (e <= 8) return ple_impl<uint8_t>(ctx, e, f, m, n, static_cast<uint8_t*>(A), lda, rank, P, Q);
  return ple_impl<uint16_t>(ctx, e, f, m, n, static_cast<uint16_t*>(A), lda, rank, P, Q);
}

}  // extern "C"
