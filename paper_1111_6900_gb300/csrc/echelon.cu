// Reduced row echelon form over GF(2^e) (Section 4.1, Algorithm 4; Section 6
// builds the echelon forms on it and on fast multiplication).
//
// Algorithm 4 takes one column at a time: the first row at or below the
// current rank r with a non-zero entry becomes the pivot row; it is scaled to
// a leading 1, moved to row r, and its multiples clear the column from every
// other row.  Here the same elimination runs by panels of W = 64 columns,
// and the work on the rest of the matrix is slice GEMMs:
//
//   1. Candidates: R = 96 rows at or below r, at first simply the next R
//      rows; in later rounds of a panel the rows with a non-zero entry in one
//      of the panel's columns that have no pivot yet, moved to rows r, r+1, ...
//   2. One CTA reduces the candidate block, column by column (first non-zero
//      candidate row), on its bit slices held in registers, to find the pivot
//      rows and columns and M^{-1} (M = the pivot rows' entries at the pivot
//      columns), which it tracks during the elimination.
//   3. The pivot rows move to rows r .. r + k - 1.  With X = M^{-1} times the
//      pivot rows (columns c0 .. n-1, one product), every row i gets
//      A[i][c0..] += A[i][pivot columns] X (one product over all m rows, the
//      multipliers copied out first): that clears the pivot columns of every
//      other row and, in characteristic 2, zeroes the pivot rows, which then
//      become X (leading 1s).
//
// A panel column may be left without a pivot while a row outside the
// candidates still has a non-zero entry there; step 1 then finds that row and
// another round runs.  The panel's pivot rows are finally put in pivot-column
// order.  Whatever rows are chosen as pivots, the result is the unique
// reduced row echelon form of A.  For random dense input the first round
// finds all W pivots (R - W spare rows), so a panel costs one read-back of
// the pivot list, the panel kernel, two products and a few copies.
#include <algorithm>
#include <numeric>
#include <vector>

#include "context.h"
#include "bitslice.cuh"
#include "rowmove.cuh"

namespace m4rie {

// trsm.cu: log / antilog tables of the field in the context: log at
// [0, 1024) (log 0 = 2(2^e - 1)), antilog at [1024, 5120), so that
// a * b = antilog[log a + log b] for all a, b.
m4rie_status ensure_field_tables(m4rie_ctx* ctx, int e, uint32_t f);

namespace {

constexpr int W = 64;         // panel columns
constexpr int R = 96;         // candidate rows per round
constexpr int LOGW = 1024;    // log table entries
constexpr int EXPW = 4096;    // antilog entries (doubled, then zeros: log 0 points there)

struct PanelOut {
  int k;            // pivots found this round
  int rows[W];      // candidate index of pivot a
  int cols[W];      // panel column of pivot a
};

// Device-side bookkeeping of the pipelined form (see echelon_pipelined): the
// panel kernel reads the rank before its panel from rr[0] and writes the rank
// after it to rr[1], the panel's pivot columns to piv[rank ..], and the new
// order of its candidate block to moves: moves[0] = cnt, moves[1 + x] = the
// candidate that goes to row rank + x (the pivot rows first, in pivot order,
// then the other candidates in order).
//
// With blk set, the candidate block is not read from A: blk holds it (R rows
// of W entries) before the previous panel's update, which the kernel applies
// itself: X's rows over this panel's columns are M_prev^{-1} (mprev, W x W)
// times the previous pivot rows there (pvn, row stride ldp), and candidate
// row x gets multp[(r + x) W + a] times X's row a, a < the previous panel's
// pivots (rr_in[0] - rr_in[-1]).
struct DevPanel {
  const int* rr_in = nullptr;
  int* rr_out = nullptr;
  int64_t* piv = nullptr;
  int* moves = nullptr;
  int64_t m = 0;
  const void* blk = nullptr;
  const void* pvn = nullptr;
  int64_t ldp = 0;
  const void* mprev = nullptr;
  const void* multp = nullptr;
};
static_assert(sizeof(PanelOut) <= kPanelHostBytes, "pinned pivot list");

// Rows i in [r, m) with a non-zero entry in a panel column not yet marked
// done (done: bit j of done[j / 64]); the first R of them (in arrival order)
// go to cand, count gets their number.
template <typename T>
__global__ void select_rows(const T* __restrict__ A, int64_t lda, int64_t m, int64_t r, int64_t c0, int wc,
                            uint64_t done0, uint64_t done1, int* __restrict__ cand, int* __restrict__ count) {
  const int64_t i = r + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const T* row = A + i * lda + c0;
  bool nz = false;
  for (int j = 0; j < wc && !nz; ++j) {
    nz = !((done0 >> j) & 1ull) && row[j] != 0;
  }
  if (nz) {
    const int idx = atomicAdd(count, 1);
    if (idx < R) cand[idx] = (int)i;
  }
}

// Step 2 on the candidate block A[r .. r+cnt)[c0 .. c0+wc) (cnt <= R): the
// pivot rows and columns and M^{-1}, from the slices of the block (Section 3.2).  Thread (row, word) of the
// 384 holds, for its candidate row, the E slices of one 32-bit word: words 0
// and 1 are the panel's 64 columns, words 2 and 3 a transform of 64 entries
// indexed by pivot order.  Column j (not done): the lowest non-pivot row with
// a non-zero entry becomes pivot number a; its transform gets coefficient 1
// at a (its own original row); every other row i with entry x_i adds
// (x_i / pv) times the pivot row, a GF(2)-linear map of the E slices (the
// columns of the matrix of multiplication by x_i / pv are (x_i / pv) x^t mod f).
// Only pivot rows are ever added into other rows, so a transform holds the
// row's combination of original pivot rows.  Pivot rows are not scaled in the
// loop (later steps never change a pivot's own entry), so at the end pivot
// row a has pv_a at its pivot column and zeros at the others, and
// M^{-1}[a][b] = pv_a^{-1} * transform[a][b].  Two barriers per column.
constexpr int BS_THREADS = 4 * R;

template <typename T, int E>
__global__ void __launch_bounds__(BS_THREADS) panel_bitsliced(const T* __restrict__ A, int64_t lda, int64_t r,
                                                              int64_t c0, int cnt, int wc, uint64_t done,
                                                              uint32_t flow, const uint16_t* __restrict__ gf,
                                                              PanelOut* __restrict__ out, T* __restrict__ minv,
                                                              int* status, DevPanel dev) {
  if (dev.rr_in) {  // pipelined form: the rank before this panel from the device
    r = *dev.rr_in;
    cnt = (int)min((int64_t)R, dev.m - r);
  }
  __shared__ uint16_t lg[LOGW];
  __shared__ uint16_t ex[EXPW];
  __shared__ uint32_t pivs[E][4];  // slices of the current pivot row
  __shared__ int cand[2];          // lowest candidate row of a column (two, used alternately)
  __shared__ uint32_t pv_s;
  __shared__ int piv_row[W], piv_col[W];
  __shared__ uint32_t piv_val[W];
  // the previous panel's update of the block (pipelined form with blk)
  __shared__ T smv[W][W];  // M_prev^{-1}, transposed: a thread per row of X reads along a row here
  constexpr int MP = W + 16 / (int)sizeof(T);  // padded multiplier rows: 16-byte aligned, no bank conflicts
  __shared__ __align__(16) T smult[R][MP];
  __shared__ uint32_t xsp[W * E * 2], xsx[W * E * 2];
  const uint32_t q = (1u << E) - 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = warp * 8 + (lane >> 2), word = lane & 3;
  // the logs of the non-zero elements and the antilogs up to 2(2^e - 1)
  for (int i = tid; i < (int)(3 * q); i += BS_THREADS) {
    if (i < (int)q) lg[i + 1] = gf[i + 1];
    else ex[i - q] = gf[LOGW + i - q];
  }
  if (tid < 2) cand[tid] = R;
  // slices of this thread's word (panel words only; transforms start at zero)
  uint32_t sl[E];
#pragma unroll
  for (int t = 0; t < E; ++t) sl[t] = 0;
  bool bad = false;
  const T* blk = static_cast<const T*>(dev.blk);
  if (word < 2 && row < cnt)
    bad = bitslice::load_word<T, E>(blk ? blk + (int64_t)row * W + 32 * word : A + (r + row) * lda + c0 + 32 * word,
                                    32 * word, 0, wc, sl);
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kStatusRange);
  if (blk) {
    const int kp = dev.rr_in[0] - dev.rr_in[-1];
    const T* mprev = static_cast<const T*>(dev.mprev);
    const T* pvn = static_cast<const T*>(dev.pvn);
#pragma unroll 4
    for (int i = tid; i < kp * W; i += BS_THREADS) smv[i % W][i / W] = mprev[i];
    if (tid < 2 * kp) {
      uint32_t gs[E];
      bitslice::load_word<T, E>(pvn + (int64_t)(tid >> 1) * dev.ldp + 32 * (tid & 1), 32 * (tid & 1), 0, wc, gs);
#pragma unroll
      for (int t = 0; t < E; ++t) xsp[((tid >> 1) * E + t) * 2 + (tid & 1)] = gs[t];
    }
    constexpr int VPR = W * (int)sizeof(T) / 16;  // 16-byte vectors per multiplier row
    const uint4* m4 = reinterpret_cast<const uint4*>(static_cast<const T*>(dev.multp) + r * W);
    uint4* d4 = reinterpret_cast<uint4*>(&smult[0][0]);
    for (int i = tid; i < cnt * VPR; i += BS_THREADS) d4[(i / VPR) * (MP * (int)sizeof(T) / 16) + i % VPR] = m4[i];
    __syncthreads();
    // X's rows over this panel's columns: X_a = sum_b M_prev^{-1}[a][b] P_b
    if (tid < 2 * kp) {
      const int a = tid >> 1, wd = tid & 1;
      uint32_t acc[E];
#pragma unroll
      for (int t = 0; t < E; ++t) acc[t] = 0;
      for (int b = 0; b < kp; ++b) {
        const uint32_t sv = smv[b][a];
        if (sv) bitslice::add_scaled<E>(acc, sv, &xsp[b * E * 2 + wd], 2, flow);
      }
#pragma unroll
      for (int t = 0; t < E; ++t) xsx[(a * E + t) * 2 + wd] = acc[t];
    }
    __syncthreads();
    // the block += its multipliers times X
    if (word < 2 && row < cnt) {
      for (int a = 0; a < kp; ++a) {
        const uint32_t sv = smult[row][a];
        if (sv) bitslice::add_scaled<E>(sl, sv, &xsx[a * E * 2 + word], 2, flow);
      }
    }
  }
  __syncthreads();

  int k = 0, my_a = -1;  // pivots so far (uniform), this row's pivot number
  int it = 0;            // columns processed (uniform): cand[it & 1] serves column it
  for (int j = 0; j < wc; ++j) {
    if ((done >> j) & 1ull) continue;
    const int wj = j >> 5, bj = j & 31;
    uint32_t x = 0;
    if (word == wj) {
#pragma unroll
      for (int t = 0; t < E; ++t) x |= ((sl[t] >> bj) & 1u) << t;
    }
    x = __shfl_sync(0xffffffffu, x, (lane & ~3) | wj);  // the entry at column j, to the row's four lanes
    const bool hit = word == wj && row < cnt && my_a < 0 && x != 0;
    const uint32_t bal = __ballot_sync(0xffffffffu, hit);
    if (lane == 0 && bal) atomicMin(&cand[it & 1], warp * 8 + ((__ffs(bal) - 1) >> 2));
    __syncthreads();
    const int p = cand[it & 1];
    // the other slot serves the next column: its last reads were before this
    // column's barrier, its next writes come after the barrier below
    if (tid == 0) cand[(it + 1) & 1] = R;
    ++it;
    if (p == R) {  // no pivot in this column among the candidates (uniform)
      __syncthreads();
      continue;
    }
    if (row == p) {
      my_a = k;
      if (word == 2 + (k >> 5)) sl[0] ^= 1u << (k & 31);  // coefficient 1 on its own original row
#pragma unroll
      for (int t = 0; t < E; ++t) pivs[t][word] = sl[t];
      if (word == 0) {
        pv_s = x;
        piv_row[k] = p;
        piv_col[k] = j;
        piv_val[k] = x;
      }
    }
    ++k;
    __syncthreads();
    if (row != p && x != 0) {
      // row += (x / pv) * pivot row, slice by slice
      uint32_t m = ex[lg[x] + q - lg[pv_s]];
#pragma unroll
      for (int t = 0; t < E; ++t) {
        const uint32_t pt = pivs[t][word];
#pragma unroll
        for (int s2 = 0; s2 < E; ++s2) sl[s2] ^= pt & (0u - ((m >> s2) & 1u));
        m = (m << 1) ^ (((m >> (E - 1)) & 1u) ? (flow | (1u << E)) : 0u);  // times x mod f
      }
    }
  }

  // M^{-1}: pivot row a's transform scaled by pv_a^{-1}
  if (my_a >= 0 && word >= 2) {
    const uint32_t linv = q - lg[piv_val[my_a]];
    for (int b0 = 0; b0 < 32; ++b0) {
      const int b = 32 * (word - 2) + b0;
      if (b >= k) break;
      uint32_t v = 0;
#pragma unroll
      for (int t = 0; t < E; ++t) v |= ((sl[t] >> b0) & 1u) << t;
      minv[my_a * W + b] = (T)(v ? ex[lg[v] + linv] : 0u);
    }
  }
  if (tid == 0) out->k = k;
  __syncthreads();
  for (int a = tid; a < k; a += BS_THREADS) {
    out->rows[a] = piv_row[a];
    out->cols[a] = piv_col[a];
  }
  if (dev.rr_in) {
    // M^{-1} as a W x W matrix: zeros outside its k x k block, so that the
    // products can always take K = W
    for (int i = tid; i < W * W; i += BS_THREADS)
      if (i / W >= k || i % W >= k) minv[i] = (T)0;
    for (int a = tid; a < k; a += BS_THREADS) dev.piv[r + a] = c0 + piv_col[a];
    if (tid == 0) {
      *dev.rr_out = (int)(r + k);
      // pivot rows to r .. r+k-1 in pivot order, the other candidates after them in order
      uint32_t used[(R + 31) / 32] = {};
      for (int a = 0; a < k; ++a) used[piv_row[a] >> 5] |= 1u << (piv_row[a] & 31);
      int next = 0;
      for (int x = 0; x < cnt; ++x) {
        int src;
        if (x < k) {
          src = piv_row[x];
        } else {
          while ((used[next >> 5] >> (next & 31)) & 1u) ++next;
          src = next++;
        }
        dev.moves[1 + x] = src;
      }
      dev.moves[0] = cnt;
    }
  }
}

template <typename T>
cudaError_t launch_panel_bitsliced(int e, const T* A, int64_t lda, int64_t r, int64_t c0, int cnt, int wc,
                                   uint64_t done, uint32_t f, const uint16_t* gf, PanelOut* out, T* minv, int* status,
                                   cudaStream_t s, const DevPanel& dev = DevPanel()) {
  const uint32_t flow = f & ((1u << e) - 1u);
#define M4RIE_PANEL_CASE(EE)                                                                                        \
  case EE:                                                                                                          \
    panel_bitsliced<T, EE><<<1, BS_THREADS, 0, s>>>(A, lda, r, c0, cnt, wc, done, flow, gf, out, minv, status, dev); \
    break;
  switch (e) {
    M4RIE_PANEL_CASE(2)
    M4RIE_PANEL_CASE(3)
    M4RIE_PANEL_CASE(4)
    M4RIE_PANEL_CASE(5)
    M4RIE_PANEL_CASE(6)
    M4RIE_PANEL_CASE(7)
    M4RIE_PANEL_CASE(8)
    M4RIE_PANEL_CASE(9)
    M4RIE_PANEL_CASE(10)
    default: return cudaErrorInvalidValue;
  }
#undef M4RIE_PANEL_CASE
  return cudaGetLastError();
}

// Multipliers of every row: mult[i][a] = A[i][c0 + cols[a]].
template <typename T>
__global__ void gather_mult(const T* __restrict__ A, int64_t lda, int64_t m, int k, int64_t c0,
                            const PanelOut* __restrict__ po, T* __restrict__ mult) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * k) return;
  const int64_t i = idx / k;
  const int a = (int)(idx % k);
  mult[i * W + a] = A[i * lda + c0 + po->cols[a]];
}

// ---------------------------------------------------------------- pipelined form
// The kernels below read the rank before the panel (rr[0]) and after it
// (rr[1]) from the device, so that every panel is queued without waiting for
// the previous one's pivot list.

// The preparation of a panel's products, reading the rank before the panel
// (rr[0]) and after it (rr[1]) and the candidate order `ord` (moves of the
// panel kernel) from the device:
//   * the candidate block's new row order, columns c0 .. c0+nt-1;
//   * the pivot block pb (W x nt): row a < k is pivot row a, the rest zero;
//   * the multipliers of every row, mult[i][a] = A[i][c0 + cols[a]] for
//     a < k, 0 above; pivot row a also gets 1 added at a, so that the
//     update A += mult X turns it into X's row a (P_a + (M_a + e_a) X = X_a
//     in characteristic 2, X = M^{-1} P);
//   * with wn > 0, blk: the next panel's candidate block (rows r + k .., the
//     next wn columns, in the new order) for the next panel kernel, which
//     applies this panel's update to it itself.
// CTA roles, in grid order:
//   * nch chunk CTAs, chunks ch0 .., each PREP_CW columns of the candidate
//     block through shared memory (chunk 0 holds this panel's and the next
//     panel's columns: it also writes the block's multipliers and blk's rows
//     inside the block);
//   * nmult CTAs of multipliers of the rows outside the block: next_only = 1,
//     only those of the next candidate block; next_only = 2, all but those;
//     0, all (these rows do not move);
//   * nblk CTAs of blk's rows outside this candidate block.
constexpr int PREP_CW = 128;
// Largest e for which the next panel's kernel applies the previous panel's
// update to its candidate block itself (its cost grows as e^2 per step).
constexpr int kPreUpdateMaxE = 4;

template <typename T>
__global__ void __launch_bounds__(256) prep_panel_dev(T* __restrict__ A, int64_t lda, int64_t m, int64_t c0,
                                                      int64_t nt, const int* __restrict__ rr,
                                                      const PanelOut* __restrict__ po, const int* __restrict__ ord,
                                                      T* __restrict__ mult, T* __restrict__ pb, int ch0, int nch,
                                                      int nmult, int next_only, T* __restrict__ blk, int wn) {
  __shared__ T stage[R][PREP_CW];
  __shared__ int so[R];
  __shared__ int scols[W];
  const int64_t r = rr[0];
  const int k = rr[1] - rr[0];
  const int cnt = ord[0];
  const int cn = (int)min((int64_t)R, m - r - k);  // rows of the next candidate block
  const int tid = threadIdx.x;
  for (int i = tid; i < k; i += 256) scols[i] = po->cols[i];
  if ((int)blockIdx.x < nch) {
    const int chunk = ch0 + (int)blockIdx.x;
    const int64_t cb = (int64_t)chunk * PREP_CW;
    const int cw = (int)min((int64_t)PREP_CW, nt - cb);
    for (int i = tid; i < cnt; i += 256) so[i] = ord[1 + i];
    // loads issued eight at a time (the loop has no dependence between iterations)
#pragma unroll 8
    for (int idx = tid; idx < cnt * PREP_CW; idx += 256) {
      const int x = idx / PREP_CW, c = idx % PREP_CW;
      if (c < cw) stage[x][c] = A[(r + x) * lda + c0 + cb + c];
    }
    __syncthreads();
    for (int idx = tid; idx < cnt * PREP_CW; idx += 256) {
      const int x = idx / PREP_CW, c = idx % PREP_CW;
      if (c < cw) A[(r + x) * lda + c0 + cb + c] = stage[so[x]][c];
    }
    for (int idx = tid; idx < W * PREP_CW; idx += 256) {
      const int a = idx / PREP_CW, c = idx % PREP_CW;
      if (c < cw) pb[(int64_t)a * nt + cb + c] = a < k ? stage[so[a]][c] : (T)0;
    }
    if (chunk == 0) {
      for (int idx = tid; idx < cnt * W; idx += 256) {
        const int x = idx / W, a = idx % W;
        T v = a < k ? stage[so[x]][scols[a]] : (T)0;
        if (a == x && a < k) v ^= (T)1;
        mult[(r + x) * W + a] = v;
      }
      if (wn > 0) {
        for (int idx = tid; idx < R * W; idx += 256) {
          const int y = idx / W, c = idx % W;
          if (y < cn && k + y < cnt) blk[idx] = c < wn ? stage[so[k + y]][W + c] : (T)0;
        }
      }
    }
    return;
  }
  __syncthreads();
  if ((int)blockIdx.x < nch + nmult) {
    const int64_t idx = ((int64_t)blockIdx.x - nch) * 256 + tid;
    int64_t i;
    if (next_only == 1) {  // the next candidate block's rows outside this one
      i = r + cnt + idx / W;
      if (i >= r + k + cn) return;
    } else {
      i = idx / W;
      if (i >= m || (i >= r && i < r + cnt)) return;
      if (next_only == 2 && i >= r + cnt && i < r + k + cn) return;
    }
    const int a = (int)(idx % W);
    mult[i * W + a] = a < k ? A[i * lda + c0 + scols[a]] : (T)0;
    return;
  }
  const int idx = ((int)blockIdx.x - nch - nmult) * 256 + tid;
  const int y = idx / W, c = idx % W;
  if (wn <= 0 || y >= cn || k + y < cnt) return;
  blk[idx] = c < wn ? A[(r + k + y) * lda + c0 + W + c] : (T)0;
}

// *flag = 1 unless every row i < r is zero left of its pivot column piv[i]
// and every row at or below r is zero (r = *rr): the pipelined pass missed
// a pivot.  Every panel clears its pivot columns in all rows, so with this
// the matrix is in reduced row echelon form.
template <typename T>
__global__ void check_echelon(const T* __restrict__ A, int64_t lda, int64_t n, const int* __restrict__ rr,
                              const int64_t* __restrict__ piv, int* __restrict__ flag) {
  const int64_t i = blockIdx.x;
  const int64_t r = *rr;
  const int64_t lim = i < r ? piv[i] : n;
  const T* row = A + i * lda;
  bool nz = false;
  for (int64_t c = threadIdx.x; c < lim; c += blockDim.x) nz |= row[c] != 0;
  if (__syncthreads_or(nz) && threadIdx.x == 0) atomicOr(flag, 1);
}

size_t ew(int e) { return rowmove::elem_bytes(e); }
using rowmove::fail;
using rowmove::move_rows;

constexpr int MOVE_SLOT = rowmove::kSlot;
static_assert(R == rowmove::kRows, "candidate blocks and move lists have the same bound");

struct Ews : rowmove::Bufs {
  int* cand = nullptr;      // [R] + count
  PanelOut* po = nullptr;
  uint8_t* minv = nullptr;  // [W][W]
  uint8_t* mult = nullptr;  // [m][W]
  uint8_t* X = nullptr;     // [W][n]
};

// Moves that bring rows want[0..] (sorted) to positions base, base+1, ...;
// the rows they displace take the vacated positions.
void placement(const std::vector<int>& want, int base, std::vector<int>& src, std::vector<int>& dst) {
  src.clear();
  dst.clear();
  const int c = (int)want.size();
  std::vector<int> vacated, displaced;
  for (int j = 0; j < c; ++j)
    if (want[j] != base + j) {
      src.push_back(want[j]);
      dst.push_back(base + j);
    }
  for (int v : want)
    if (v >= base + c) vacated.push_back(v);
  for (int t = base; t < base + c; ++t)
    if (!std::binary_search(want.begin(), want.end(), t)) displaced.push_back(t);
  for (size_t i = 0; i < displaced.size(); ++i) {
    src.push_back(displaced[i]);
    dst.push_back(vacated[i]);
  }
}

// The reduced row echelon form with every panel queued up front: the panel
// kernels keep the rank and the candidate order on the device, and the
// products always take K = W (M^{-1} is zero outside its k x k block, so the
// unused multiplier columns add nothing).  Per panel: one preparation
// kernel; then the next panel's kernel on the side stream, from a snapshot of
// its candidate block to which it applies this panel's update itself, beside
// this panel's two products (X and the update).  The pivot list is read back
// once, at the end.  Each panel takes one round with the next R rows as
// candidates, so a column whose only non-zero entries lie below them gets no
// pivot.  A final check flags that case (*complete = false);
// the matrix is then row-equivalent to the input, and the caller finishes
// it with echelon_impl (the reduced form is unique).
template <typename T>
m4rie_status echelon_pipelined(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, T* A, int64_t lda,
                               int64_t* rank, int64_t* pivots, bool* complete) {
  *complete = false;
  const size_t w = ew(e);
  const int P = (int)ceil_div(n, W);
  const size_t sz_po = round_up((int64_t)sizeof(PanelOut), 256);
  const size_t sz_minv = round_up((int64_t)((size_t)W * W * w), 256);
  const size_t sz_mult = round_up((int64_t)((size_t)m * W * w), 256);
  const size_t sz_X = round_up((int64_t)((size_t)W * n * w), 256);
  const size_t sz_rr = round_up((int64_t)(sizeof(int) * (P + 2)), 256);
  const size_t sz_piv = round_up((int64_t)(sizeof(int64_t) * std::min(m, n)), 256);
  const size_t sz_mv = round_up((int64_t)(sizeof(int) * (1 + 2 * R) + 64), 256);
  const size_t sz_blk = round_up((int64_t)((size_t)R * W * w), 256);
  const size_t total = sz_po + 2 * sz_minv + sz_mult + 2 * sz_X + sz_rr + sz_piv + sz_mv + sz_blk;
  cudaError_t err;
  if (total > ctx->ews_bytes) {
    if ((err = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return fail(ctx, err);
    if (ctx->ews) cudaFree(ctx->ews);
    ctx->ews = nullptr;
    ctx->ews_bytes = 0;
    if (cudaMalloc(&ctx->ews, total) != cudaSuccess) {
      cudaGetLastError();
      ctx->last_error = "echelon workspace allocation failed";
      return M4RIE_ERR_NOMEM;
    }
    ctx->ews_bytes = total;
  }
  if ((err = rowmove::ensure_side(ctx)) != cudaSuccess) return fail(ctx, err);
  uint8_t* base = static_cast<uint8_t*>(ctx->ews);
  PanelOut* po = reinterpret_cast<PanelOut*>(base);
  T* minv2[2] = {reinterpret_cast<T*>(base + sz_po), reinterpret_cast<T*>(base + sz_po + sz_minv)};
  uint8_t* b2 = base + sz_po + 2 * sz_minv;
  T* mult = reinterpret_cast<T*>(b2);
  T* X = reinterpret_cast<T*>(b2 + sz_mult);
  T* pb = reinterpret_cast<T*>(b2 + sz_mult + sz_X);
  int* rr = reinterpret_cast<int*>(b2 + sz_mult + 2 * sz_X);
  int64_t* piv = reinterpret_cast<int64_t*>(b2 + sz_mult + 2 * sz_X + sz_rr);
  int* moves = reinterpret_cast<int*>(b2 + sz_mult + 2 * sz_X + sz_rr + sz_piv);
  T* blk = reinterpret_cast<T*>(b2 + sz_mult + 2 * sz_X + sz_rr + sz_piv + sz_mv);
  int* flag = moves + 1 + 2 * R;
  if ((err = cudaMemsetAsync(rr, 0, sizeof(int), ctx->stream)) != cudaSuccess ||
      (err = cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream)) != cudaSuccess)
    return fail(ctx, err);
  cudaStream_t st = ctx->stream;
  for (int p = 0; p < P; ++p) {
    const int64_t c0 = (int64_t)p * W, nt = n - c0;
    const int wc = (int)std::min<int64_t>(W, nt);
    const bool next = p + 1 < P;
    const bool pre = next && e <= kPreUpdateMaxE;
    const int wn = next ? (int)std::min<int64_t>(W, n - c0 - W) : 0;
    T* minv = minv2[p & 1];  // this panel's M^{-1}; the next panel kernel writes the other one
    if (p == 0) {
      DevPanel dv;
      dv.rr_in = rr;
      dv.rr_out = rr + 1;
      dv.piv = piv;
      dv.moves = moves;
      dv.m = m;
      if ((err = launch_panel_bitsliced<T>(e, A, lda, 0, c0, 0, wc, 0, f, ctx->d_gf, po, minv, ctx->d_status, st,
                                           dv)) != cudaSuccess)
        return fail(ctx, err);
      ++ctx->launches;
    } else if ((err = cudaStreamWaitEvent(st, ctx->ech_ev[1], 0)) != cudaSuccess) {
      return fail(ctx, err);
    }
    // 1. the candidate block in its new order, the pivot block, the
    // multipliers, the next panel's candidate block: with the look-ahead,
    // what the next panel's kernel needs in a first small launch
    const int nchunks = (int)ceil_div(nt, PREP_CW);
    const int nmult_all = (int)ceil_div(m * W, 256);
    const int nblk = pre ? (int)ceil_div(R * W, 256) : 0;
    prep_panel_dev<T><<<(unsigned)(nchunks + nmult_all + nblk), 256, 0, st>>>(
        A, lda, m, c0, nt, rr + p, po, moves, mult, pb, 0, nchunks, nmult_all, 0, blk, pre ? wn : 0);
    ++ctx->launches;
    DevPanel dn;  // the next panel's kernel
    dn.rr_in = rr + p + 1;
    dn.rr_out = rr + p + 2;
    dn.piv = piv;
    dn.moves = moves;
    dn.m = m;
    // 2. (e <= kPreUpdateMaxE) the next panel's kernel on the side stream: it
    // applies this panel's update to its candidate block itself, so it
    // waits for neither step 3 nor 4
    if (pre) {
      DevPanel dv = dn;
      dv.blk = blk;
      dv.pvn = pb + W;
      dv.ldp = nt;
      dv.mprev = minv;
      dv.multp = mult;
      if ((err = cudaEventRecord(ctx->ech_ev[0], st)) != cudaSuccess ||
          (err = cudaStreamWaitEvent(ctx->ech_side, ctx->ech_ev[0], 0)) != cudaSuccess ||
          (err = launch_panel_bitsliced<T>(e, A, lda, 0, c0 + W, 0, wn, 0, f, ctx->d_gf, po, minv2[(p + 1) & 1],
                                           ctx->d_status, ctx->ech_side, dv)) != cudaSuccess ||
          (err = cudaEventRecord(ctx->ech_ev[1], ctx->ech_side)) != cudaSuccess)
        return fail(ctx, err);
      ++ctx->launches;
    }
    // 3. X = M^{-1} (pivot rows); 4. A[:, c0..] += mult X, which also makes
    // the pivot rows X's rows.  Larger fields, where the block's update costs
    // the one-CTA kernel more than a product: the next panel's columns first,
    // then its kernel on the side stream beside the rest.
    m4rie_status s2 = run_gemm(ctx, e, f, W, nt, W, Mats{minv, W, pb, nt, X, nt}, 0);
    if (s2 != M4RIE_OK) return s2;
    const int64_t n1 = next && !pre && nt > 2 * W ? 2 * W : nt;
    if ((s2 = run_gemm(ctx, e, f, m, n1, W, Mats{mult, W, X, nt, A + c0, lda}, 1)) != M4RIE_OK) return s2;
    if (next && !pre) {
      if ((err = cudaEventRecord(ctx->ech_ev[0], st)) != cudaSuccess ||
          (err = cudaStreamWaitEvent(ctx->ech_side, ctx->ech_ev[0], 0)) != cudaSuccess ||
          (err = launch_panel_bitsliced<T>(e, A, lda, 0, c0 + W, 0, wn, 0, f, ctx->d_gf, po, minv2[(p + 1) & 1],
                                           ctx->d_status, ctx->ech_side, dn)) != cudaSuccess ||
          (err = cudaEventRecord(ctx->ech_ev[1], ctx->ech_side)) != cudaSuccess)
        return fail(ctx, err);
      ++ctx->launches;
    }
    if (n1 < nt &&
        (s2 = run_gemm(ctx, e, f, m, nt - n1, W, Mats{mult, W, X + n1, nt, A + c0 + n1, lda}, 1)) != M4RIE_OK)
      return s2;
    if ((err = cudaGetLastError()) != cudaSuccess) return fail(ctx, err);
  }
  check_echelon<T><<<(unsigned)m, 256, 0, st>>>(A, lda, n, rr + P, piv, flag);
  ++ctx->launches;
  int h[2] = {0, 0};
  if ((err = cudaMemcpyAsync(&h[0], flag, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (err = cudaMemcpyAsync(&h[1], rr + P, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (err = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(ctx, err);
  if (h[0]) return M4RIE_OK;  // a pivot was missed: *complete stays false
  const int64_t r = h[1];
  if (r < 0 || r > std::min(m, n)) {
    ctx->last_error = "echelon form: inconsistent rank on the device";
    return M4RIE_ERR_CUDA;
  }
  if (pivots && r > 0 &&
      (err = cudaMemcpy(pivots, piv, sizeof(int64_t) * (size_t)r, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return fail(ctx, err);
  if (rank) *rank = r;
  *complete = true;
  return M4RIE_OK;
}

template <typename T>
m4rie_status echelon_impl(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, T* A, int64_t lda, int64_t* rank,
                          int64_t* pivots) {
  const size_t w = ew(e);
  const size_t sz_cand = round_up((int64_t)(sizeof(int) * (R + 1 + 2 * MOVE_SLOT)), 256);
  const size_t sz_po = round_up((int64_t)sizeof(PanelOut), 256);
  const size_t sz_minv = round_up((int64_t)((size_t)W * W * w), 256);
  const size_t sz_mult = round_up((int64_t)((size_t)m * W * w), 256);
  const size_t sz_X = round_up((int64_t)((size_t)W * n * w), 256);
  const size_t sz_tmp = round_up((int64_t)((size_t)2 * R * n * w), 256);
  const size_t total = sz_cand + sz_po + sz_minv + sz_mult + sz_X + sz_tmp;
  cudaError_t err;
  if (total > ctx->ews_bytes) {
    if ((err = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return fail(ctx, err);
    if (ctx->ews) cudaFree(ctx->ews);
    ctx->ews = nullptr;
    ctx->ews_bytes = 0;
    if (cudaMalloc(&ctx->ews, total) != cudaSuccess) {
      cudaGetLastError();
      ctx->last_error = "echelon workspace allocation failed";
      return M4RIE_ERR_NOMEM;
    }
    ctx->ews_bytes = total;
  }
  if (!ctx->ews_host && cudaMallocHost(&ctx->ews_host, sizeof(int) * 2 * MOVE_SLOT) != cudaSuccess) {
    cudaGetLastError();
    ctx->ews_host = nullptr;
    ctx->last_error = "pinned host buffer allocation failed";
    return M4RIE_ERR_NOMEM;
  }
  Ews ws;
  uint8_t* base = static_cast<uint8_t*>(ctx->ews);
  ws.cand = reinterpret_cast<int*>(base);
  ws.moves = ws.cand + R + 1;
  ws.po = reinterpret_cast<PanelOut*>(base + sz_cand);
  ws.minv = base + sz_cand + sz_po;
  ws.mult = ws.minv + sz_minv;
  ws.X = ws.mult + sz_mult;
  ws.tmp = ws.X + sz_X;
  ws.host = ctx->ews_host;
  int* d_count = ws.cand + R;


  // look-ahead: the next panel's factorisation on a side stream (non-blocking,
  // ordered against ctx->stream by events), its pivot list into pinned memory
  if ((err = rowmove::ensure_side(ctx)) != cudaSuccess) return fail(ctx, err);
  PanelOut* hpo_next = static_cast<PanelOut*>(ctx->ech_po_host);
  bool ahead = false;  // the current panel's round-0 factorisation was launched by the previous panel

  std::vector<int64_t> piv_cols;
  int64_t r = 0;
  std::vector<int> src, dst, hc(R + 1);
  PanelOut hpo;
  for (int64_t c0 = 0; c0 < n && r < m; c0 += W) {
    const int wc = (int)std::min<int64_t>(W, n - c0);
    const int64_t nt = n - c0;
    uint64_t done = 0;
    const int64_t r_panel = r;
    std::vector<int64_t> panel_cols;  // pivot column of rows r_panel.. in row order
    bool reordered = false;
    for (int round = 0; r < m; ++round) {
      // 1. candidates: the next R rows, or (later rounds) rows with a non-zero open entry
      int cnt;
      if (round == 0) {
        cnt = (int)std::min<int64_t>(R, m - r);
      } else {
        if ((err = cudaMemsetAsync(d_count, 0, sizeof(int), ctx->stream)) != cudaSuccess) return fail(ctx, err);
        select_rows<T><<<(unsigned)ceil_div(m - r, 256), 256, 0, ctx->stream>>>(A, lda, m, r, c0, wc, done, 0,
                                                                              ws.cand, d_count);
        ++ctx->launches;
        if ((err = cudaMemcpyAsync(hc.data(), ws.cand, sizeof(int) * (R + 1), cudaMemcpyDeviceToHost,
                                   ctx->stream)) != cudaSuccess ||
            (err = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
          return fail(ctx, err);
        cnt = std::min(hc[R], R);
        if (cnt == 0) break;
        std::vector<int> want(hc.begin(), hc.begin() + cnt);
        std::sort(want.begin(), want.end());
        placement(want, (int)r, src, dst);
        if ((err = move_rows<T>(ctx, ws, 0, A, lda, c0, nt, src, dst)) != cudaSuccess) return fail(ctx, err);
      }
      // 2. pivots of the candidate block and M^{-1}
      if (round == 0 && ahead) {
        // launched on the side stream while the previous panel's update ran
        if ((err = cudaEventSynchronize(ctx->ech_ev[1])) != cudaSuccess ||
            (err = cudaStreamWaitEvent(ctx->stream, ctx->ech_ev[1], 0)) != cudaSuccess)
          return fail(ctx, err);
        hpo = *hpo_next;
        ahead = false;
      } else {
        if ((err = launch_panel_bitsliced<T>(e, A, lda, r, c0, cnt, wc, done, f, ctx->d_gf, ws.po,
                                             reinterpret_cast<T*>(ws.minv), ctx->d_status, ctx->stream)) !=
            cudaSuccess)
          return fail(ctx, err);
        ++ctx->launches;
        if ((err = cudaMemcpyAsync(&hpo, ws.po, sizeof(PanelOut), cudaMemcpyDeviceToHost, ctx->stream)) !=
                cudaSuccess ||
            (err = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
          return fail(ctx, err);
      }
      const int k = hpo.k;
      if (k <= 0) {
        if (round == 0) continue;  // no pivot among the next R rows: search all rows
        break;                     // cannot happen: a candidate row has a non-zero open entry
      }
      // 3. pivot rows to r .. r+k-1, the other candidates after them
      {
        std::vector<char> used(cnt, 0);
        std::vector<int> order;
        for (int a = 0; a < k; ++a) {
          used[hpo.rows[a]] = 1;
          order.push_back((int)r + hpo.rows[a]);
        }
        for (int i = 0; i < cnt; ++i)
          if (!used[i]) order.push_back((int)r + i);
        src.clear();
        dst.clear();
        for (int i = 0; i < cnt; ++i)
          if (order[i] != (int)r + i) {
            src.push_back(order[i]);
            dst.push_back((int)r + i);
          }
        if ((err = move_rows<T>(ctx, ws, 1, A, lda, c0, nt, src, dst)) != cudaSuccess) return fail(ctx, err);
      }
      // multipliers of every row, read before the update
      gather_mult<T><<<(unsigned)ceil_div(m * k, 256), 256, 0, ctx->stream>>>(A, lda, m, k, c0, ws.po,
                                                                           reinterpret_cast<T*>(ws.mult));
      ++ctx->launches;
      // X = M^{-1} (pivot rows, columns c0..); A[:, c0..] += mult X; pivot rows = X
      T* Ar = A + r * lda + c0;
      m4rie_status st = run_gemm(ctx, e, f, k, nt, k, Mats{ws.minv, W, Ar, lda, ws.X, nt}, 0);
      if (st != M4RIE_OK) return st;
      uint64_t done_after = done;
      for (int a = 0; a < k; ++a) done_after |= 1ull << hpo.cols[a];
      const bool last = __builtin_popcountll(done_after) == wc || r + k >= m;
      // Look-ahead (last round of a panel, with a next panel and candidates for
      // it): update this panel's and the next panel's columns first, start the
      // next panel's factorisation on the side stream, then update the rest.
      const int64_t r_next = r + k, c_next = c0 + W;
      const bool look = last && c_next < n && r_next < m && nt > 2 * W;
      const int64_t n1 = look ? 2 * W : nt;
      if ((st = run_gemm(ctx, e, f, m, n1, k, Mats{ws.mult, W, ws.X, nt, A + c0, lda}, 1)) != M4RIE_OK) return st;
      if (look) {
        const int cnt_next = (int)std::min<int64_t>(R, m - r_next);
        const int wc_next = (int)std::min<int64_t>(W, n - c_next);
        if ((err = cudaEventRecord(ctx->ech_ev[0], ctx->stream)) != cudaSuccess ||
            (err = cudaStreamWaitEvent(ctx->ech_side, ctx->ech_ev[0], 0)) != cudaSuccess ||
            (err = launch_panel_bitsliced<T>(e, A, lda, r_next, c_next, cnt_next, wc_next, 0, f, ctx->d_gf, ws.po,
                                             reinterpret_cast<T*>(ws.minv), ctx->d_status, ctx->ech_side)) !=
                cudaSuccess ||
            (err = cudaMemcpyAsync(hpo_next, ws.po, sizeof(PanelOut), cudaMemcpyDeviceToHost, ctx->ech_side)) !=
                cudaSuccess ||
            (err = cudaEventRecord(ctx->ech_ev[1], ctx->ech_side)) != cudaSuccess)
          return fail(ctx, err);
        ++ctx->launches;
        ahead = true;
        if ((st = run_gemm(ctx, e, f, m, nt - n1, k, Mats{ws.mult, W, ws.X + n1 * w, nt, A + c0 + n1, lda}, 1)) !=
            M4RIE_OK)
          return st;
      }
      if ((err = cudaMemcpy2DAsync(Ar, (size_t)lda * w, ws.X, (size_t)nt * w, (size_t)nt * w, (size_t)k,
                                   cudaMemcpyDeviceToDevice, ctx->stream)) != cudaSuccess)
        return fail(ctx, err);
      for (int a = 0; a < k; ++a) {
        const int j = hpo.cols[a];
        done |= 1ull << j;
        if (!panel_cols.empty() && c0 + j < panel_cols.back()) reordered = true;
        panel_cols.push_back(c0 + j);
      }
      r += k;
      if (__builtin_popcountll(done) == wc) break;
    }
    if (reordered) {
      // pivot rows of this panel in pivot-column order
      std::vector<int> idx(panel_cols.size());
      std::iota(idx.begin(), idx.end(), 0);
      std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return panel_cols[a] < panel_cols[b]; });
      src.clear();
      dst.clear();
      std::vector<int64_t> sorted_cols;
      for (size_t i = 0; i < idx.size(); ++i) {
        sorted_cols.push_back(panel_cols[idx[i]]);
        if (idx[i] != (int)i) {
          src.push_back((int)(r_panel + idx[i]));
          dst.push_back((int)(r_panel + i));
        }
      }
      if ((err = move_rows<T>(ctx, ws, 0, A, lda, c0, nt, src, dst)) != cudaSuccess) return fail(ctx, err);
      panel_cols = sorted_cols;
    }
    piv_cols.insert(piv_cols.end(), panel_cols.begin(), panel_cols.end());
  }
  if (ahead && (err = cudaEventSynchronize(ctx->ech_ev[1])) != cudaSuccess) return fail(ctx, err);
  if ((err = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return fail(ctx, err);
  if (rank) *rank = r;
  if (pivots)
    for (int64_t i = 0; i < r; ++i) pivots[i] = piv_cols[i];
  return M4RIE_OK;
}

}  // namespace
}  // namespace m4rie

using namespace m4rie;

extern "C" {

m4rie_status m4rie_echelonize(m4rie_ctx* ctx, int e, uint32_t f, int64_t m, int64_t n, void* A, int64_t lda,
                              int64_t* rank, int64_t* pivots) {
  if (!ctx) return M4RIE_ERR_ARG;
  m4rie_status st = m4rie_validate(e, f, 0, 0, 0, nullptr, nullptr, nullptr);
  if (st != M4RIE_OK) return st;
  if (m < 0 || n < 0 || m > (1ll << 31) - 1 || n > (1ll << 31) || lda < n || (m > 0 && n > 0 && !A)) return M4RIE_ERR_ARG;
  if (rank) *rank = 0;
  if (m == 0 || n == 0) return M4RIE_OK;
  if ((st = ensure_field_tables(ctx, e, f)) != M4RIE_OK) return st;
  // The pipelined form when the rank cannot run out of rows long before the
  // last panel; a missed pivot, or a wide matrix, takes the form that reads
  // each panel's pivot list back.
  if (n <= m + W) {
    bool complete = false;
    st = e <= 8 ? echelon_pipelined<uint8_t>(ctx, e, f, m, n, static_cast<uint8_t*>(A), lda, rank, pivots, &complete)
                : echelon_pipelined<uint16_t>(ctx, e, f, m, n, static_cast<uint16_t*>(A), lda, rank, pivots, &complete);
    if (st != M4RIE_OK || complete) return st;
  }
  if (e <= 8) return echelon_impl<uint8_t>(ctx, e, f, m, n, static_cast<uint8_t*>(A), lda, rank, pivots);
  return echelon_impl<uint16_t>(ctx, e, f, m, n, static_cast<uint16_t*>(A), lda, rank, pivots);
}

}  // extern "C"
