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
//   2. One CTA reduces the candidate block in shared memory, column by
//      column (first non-zero candidate row), to find the pivot rows and
//      columns, and inverts M = the pivot rows' entries at the pivot columns.
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
constexpr int PANEL_THREADS = 4 * R;  // 4 threads per candidate row, every 4th column each
// Shared row strides (u16 entries): an odd number of 32-bit words, so that the
// 8 rows a warp works on fall in different banks.
constexpr int BP = W + 2;          // candidate block [R][BP]
constexpr int GP = 2 * W + 2;      // [M | I] system [W][GP]

struct PanelOut {
  int k;            // pivots found this round
  int rows[W];      // candidate index of pivot a
  int cols[W];      // panel column of pivot a
};

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

// Row moves (columns c0 .. n-1): tmp[j] = A[src_j], then A[dst_j] = tmp[j].
template <typename T>
__global__ void gather_rows(const T* __restrict__ A, int64_t lda, int64_t c0, int64_t nt, const int* __restrict__ src,
                            T* __restrict__ tmp) {
  const int j = blockIdx.y;
  const T* s = A + (int64_t)src[j] * lda + c0;
  T* d = tmp + (int64_t)j * nt;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nt; c += (int64_t)gridDim.x * blockDim.x)
    d[c] = s[c];
}

template <typename T>
__global__ void scatter_rows(T* __restrict__ A, int64_t lda, int64_t c0, int64_t nt, const int* __restrict__ dst,
                             const T* __restrict__ tmp) {
  const int j = blockIdx.y;
  T* d = A + (int64_t)dst[j] * lda + c0;
  const T* s = tmp + (int64_t)j * nt;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nt; c += (int64_t)gridDim.x * blockDim.x)
    d[c] = s[c];
}

// Step 2 on the candidate block A[r .. r+cnt)[c0 .. c0+wc) (cnt <= R): find
// the pivots (columns in order, skipping done ones; the first candidate row
// not yet a pivot with a non-zero entry after the previous eliminations) and
// write M^{-1} (k x k, row stride W) to minv.  Entries >= 2^e set the range
// flag and are used by their low e bits.
template <typename T>
__global__ void __launch_bounds__(PANEL_THREADS) panel_factor(int e, const T* __restrict__ A, int64_t lda, int64_t r,
                                                              int64_t c0, int cnt, int wc, uint64_t done0,
                                                              uint64_t done1, const uint16_t* __restrict__ gf,
                                                              PanelOut* __restrict__ out, T* __restrict__ minv,
                                                              int* status) {
  extern __shared__ uint16_t sh[];
  uint16_t* lg = sh;
  uint16_t* ex = sh + LOGW;
  uint16_t* blk = ex + EXPW;  // [R][BP], later [W][GP] for the inversion
  __shared__ int piv_row[W], piv_col[W], is_piv[R];
  __shared__ uint16_t plg[2 * W];  // logs of the current pivot row
  __shared__ int sel, kk;
  const uint32_t q = (1u << e) - 1;
  const int tid = threadIdx.x;
  for (int i = tid; i < LOGW + EXPW; i += PANEL_THREADS) sh[i] = gf[i];
  bool bad = false;
  for (int idx = tid; idx < R * W; idx += PANEL_THREADS) {
    const int i = idx / W, j = idx % W;
    uint32_t v = 0;
    if (i < cnt && j < wc) {
      v = A[(r + i) * lda + c0 + j];
      bad |= v > q;
      v &= q;
    }
    blk[i * BP + j] = (uint16_t)v;
  }
  for (int i = tid; i < R; i += PANEL_THREADS) is_piv[i] = 0;
  (void)done1;
  if (tid == 0) kk = 0;
  if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(status, kStatusRange);
  __syncthreads();

  const int row = tid >> 2, part = tid & 3;  // this thread: row `row`, columns part, part + 4, ...
  uint16_t* br = blk + row * BP;
  for (int j = 0; j < wc; ++j) {
    if ((done0 >> j) & 1ull) continue;
    if (tid == 0) sel = R;
    __syncthreads();
    {
      // lowest candidate row (not yet a pivot) with a non-zero entry: a
      // ballot per warp (8 rows), then one atomic per warp
      const bool hit = part == 0 && row < cnt && !is_piv[row] && br[j] != 0;
      const uint32_t bal = __ballot_sync(0xffffffffu, hit);
      if ((tid & 31) == 0 && bal) atomicMin(&sel, (tid + __ffs(bal) - 1) >> 2);
    }
    __syncthreads();
    const int p = sel;
    if (p == R) continue;  // no pivot in this column among the candidates
    // scale the pivot row to a leading 1 (its entries left of j are zero),
    // one thread per column, and keep the logs of its entries
    {
      const uint32_t ld = q - lg[blk[p * BP + j]];  // log of the inverse pivot
      __syncthreads();                               // every thread has read the pivot
      if (tid < W) {
        const uint32_t v = ex[lg[blk[p * BP + tid]] + ld];
        blk[p * BP + tid] = (uint16_t)v;
        plg[tid] = lg[v];
      }
    }
    __syncthreads();
    // clear column j from every other candidate row (the pivot row is zero
    // left of j, and log 0 leads to a zero product)
    const uint32_t x = row != p && row < cnt ? br[j] : 0u;
    __syncwarp();
    if (x) {
      const uint32_t lx = lg[x];
#pragma unroll
      for (int i = 0; i < W / 4; ++i) {
        const int c = part + 4 * i;
        br[c] ^= ex[plg[c] + lx];
      }
    }
    if (tid == 0) {
      is_piv[p] = 1;
      piv_row[kk] = p;
      piv_col[kk] = j;
      ++kk;
    }
    __syncthreads();
  }
  const int k = kk;

  // M^{-1} by Gauss-Jordan on [M | I] (M invertible: k pivots were found);
  // thread (row, part) owns row `row` and columns part, part + 4, ... of the
  // k x 2k system (M in columns 0 .. W-1, I in W .. 2W-1), row stride GP.
  uint16_t* g = blk;
  __syncthreads();
  for (int idx = tid; idx < W * 2 * W; idx += PANEL_THREADS) {
    const int a = idx / (2 * W), b = idx % (2 * W);
    uint32_t v = 0;
    if (a < k && b < k) v = (uint32_t)A[(r + piv_row[a]) * lda + c0 + piv_col[b]] & q;
    else if (a < k && b >= W && b - W == a) v = 1;
    g[a * GP + b] = (uint16_t)v;
  }
  __syncthreads();
  uint16_t* gr = g + row * GP;
  for (int t = 0; t < k; ++t) {
    if (tid == 0) sel = W;
    __syncthreads();
    {
      const bool hit = part == 0 && row >= t && row < k && gr[t] != 0;
      const uint32_t bal = __ballot_sync(0xffffffffu, hit);
      if ((tid & 31) == 0 && bal) atomicMin(&sel, (tid + __ffs(bal) - 1) >> 2);
    }
    __syncthreads();
    const int p = sel;  // exists: M is invertible
    // swap rows p and t (the 4 threads of row t each swap their columns)
    if (row == t && p != t) {
      uint16_t* rp = g + p * GP;
      for (int c = part; c < 2 * W; c += 4) {
        const uint16_t s = gr[c];
        gr[c] = rp[c];
        rp[c] = s;
      }
    }
    __syncthreads();
    {
      const uint32_t ld = q - lg[g[t * GP + t]];
      __syncthreads();  // every thread has read the pivot
      if (tid < 2 * W) {
        const uint32_t v = ex[lg[g[t * GP + tid]] + ld];
        g[t * GP + tid] = (uint16_t)v;
        plg[tid] = lg[v];
      }
    }
    __syncthreads();
    const uint32_t x = row != t && row < k ? gr[t] : 0u;
    __syncwarp();
    if (x) {
      const uint32_t lx = lg[x];
#pragma unroll
      for (int i = 0; i < 2 * W / 4; ++i) {
        const int c = part + 4 * i;
        gr[c] ^= ex[plg[c] + lx];
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < k * W; idx += PANEL_THREADS) {
    const int a = idx / W, b = idx % W;
    minv[idx] = b < k ? (T)g[a * GP + W + b] : (T)0;
  }
  if (tid == 0) out->k = k;
  for (int a = tid; a < k; a += PANEL_THREADS) {
    out->rows[a] = piv_row[a];
    out->cols[a] = piv_col[a];
  }
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

size_t ew(int e) { return e <= 8 ? 1 : 2; }

constexpr int MOVE_SLOT = 4 * R;  // ints per pinned slot: up to 2R (src, dst) pairs

struct Ews {
  int* cand = nullptr;      // [R] + count
  int* moves = nullptr;     // device: two slots of [src | dst]
  PanelOut* po = nullptr;
  uint8_t* minv = nullptr;  // [W][W]
  uint8_t* mult = nullptr;  // [m][W]
  uint8_t* X = nullptr;     // [W][n]
  uint8_t* tmp = nullptr;   // [2R][n]
  int* host = nullptr;      // pinned: two slots of [src | dst]
};

m4rie_status fail(m4rie_ctx* ctx, cudaError_t err) {
  ctx->last_error = cudaGetErrorString(err);
  return M4RIE_ERR_CUDA;
}

// Row moves src[j] -> dst[j] of columns c0 .. n-1 through tmp, the lists
// staged in pinned slot `slot`.  A slot is written again only after a later
// read-back has synchronized the stream, so no wait is needed here.
template <typename T>
cudaError_t move_rows(m4rie_ctx* ctx, const Ews& w, int slot, T* A, int64_t lda, int64_t c0, int64_t nt,
                      const std::vector<int>& src, const std::vector<int>& dst) {
  const int nm = (int)src.size();
  if (nm == 0 || nt == 0) return cudaSuccess;
  int* h = w.host + slot * MOVE_SLOT;
  int* d = w.moves + slot * MOVE_SLOT;
  std::copy(src.begin(), src.end(), h);
  std::copy(dst.begin(), dst.end(), h + nm);
  cudaError_t err = cudaMemcpyAsync(d, h, sizeof(int) * 2 * nm, cudaMemcpyHostToDevice, ctx->stream);
  if (err != cudaSuccess) return err;
  const dim3 grid((unsigned)std::min<int64_t>(ceil_div(nt, 256), 64), (unsigned)nm);
  gather_rows<T><<<grid, 256, 0, ctx->stream>>>(A, lda, c0, nt, d, reinterpret_cast<T*>(w.tmp));
  scatter_rows<T><<<grid, 256, 0, ctx->stream>>>(A, lda, c0, nt, d + nm, reinterpret_cast<const T*>(w.tmp));
  ctx->launches += 2;
  return cudaGetLastError();
}

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

  const size_t panel_smem = (size_t)(LOGW + EXPW + std::max(R * BP, W * GP)) * sizeof(uint16_t);
  if ((err = cudaFuncSetAttribute(panel_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem)) !=
      cudaSuccess)
    return fail(ctx, err);

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
      panel_factor<T><<<1, PANEL_THREADS, panel_smem, ctx->stream>>>(e, A, lda, r, c0, cnt, wc, done, 0, ctx->d_gf,
                                                                    ws.po, reinterpret_cast<T*>(ws.minv),
                                                                    ctx->d_status);
      ++ctx->launches;
      if ((err = cudaMemcpyAsync(&hpo, ws.po, sizeof(PanelOut), cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess ||
          (err = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
        return fail(ctx, err);
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
      if ((st = run_gemm(ctx, e, f, m, nt, k, Mats{ws.mult, W, ws.X, nt, A + c0, lda}, 1)) != M4RIE_OK) return st;
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
  if (m < 0 || n < 0 || m > (1ll << 31) - 1 || n > (1ll << 31) || lda < n || (m * n && !A)) return M4RIE_ERR_ARG;
  if (rank) *rank = 0;
  if (m == 0 || n == 0) return M4RIE_OK;
  if ((st = ensure_field_tables(ctx, e, f)) != M4RIE_OK) return st;
  if (e <= 8) return echelon_impl<uint8_t>(ctx, e, f, m, n, static_cast<uint8_t*>(A), lda, rank, pivots);
  return echelon_impl<uint16_t>(ctx, e, f, m, n, static_cast<uint16_t*>(A), lda, rank, pivots);
}

}  // extern "C"
