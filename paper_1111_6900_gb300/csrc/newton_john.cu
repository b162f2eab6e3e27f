// Newton-John multiplication (Section 4, Algorithms 2 and 3) on the packed
// representation (Section 3.1): tile plan and dispatch, and the conversions
// between element arrays and packed rows.  The kernel is in nj_kernel.cuh.
#include "nj_kernel.cuh"

namespace m4rie {
using nj::flag_range;
using nj::kWarps;
namespace {

int nj_chunk(int e) {
  switch (e) {
    case 2: return nj::Nj<2>::KT;
    case 3: return nj::Nj<3>::KT;
    case 4: return nj::Nj<4>::KT;
    case 5: return nj::Nj<5>::KT;
    case 6: return nj::Nj<6>::KT;
    case 7: return nj::Nj<7>::KT;
    case 8: return nj::Nj<8>::KT;
    case 9: return nj::Nj<9>::KT;
    case 10: return nj::Nj<10>::KT;
  }
  return 0;
}

// ---------------------------------------------------------------- conversions

// One thread per 32-bit word of the packed output (including the padding
// words up to ld32): fields from the elements, zero beyond cols.
__global__ void to_packed_kernel(int e, int64_t rows, int64_t cols, const void* __restrict__ X, int64_t ldx,
                                 int elem_bytes, uint32_t* __restrict__ out, int64_t ld32, int* status) {
  const int W = packed_width(e), P = 32 / W;
  const uint32_t em = (1u << e) - 1u;
  bool bad = false;
  const int64_t total = rows * ld32;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / ld32, wc = idx - r * ld32;
    uint32_t w = 0;
    for (int j = 0; j < P; ++j) {
      const int64_t c = wc * P + j;
      if (c >= cols) break;
      const uint32_t x = elem_bytes == 1 ? static_cast<const uint8_t*>(X)[r * ldx + c]
                                         : static_cast<const uint16_t*>(X)[r * ldx + c];
      bad |= x > em;
      w |= (x & em) << (j * W);
    }
    out[idx] = w;
  }
  flag_range(status, bad);
}

// One thread per 32-bit word holding at least one of the cols fields.
__global__ void from_packed_kernel(int e, int64_t rows, int64_t cols, const uint32_t* __restrict__ in, int64_t ld32,
                                   void* __restrict__ X, int64_t ldx, int elem_bytes) {
  const int W = packed_width(e), P = 32 / W;
  const uint32_t em = (1u << e) - 1u;
  const int64_t nw = (cols + P - 1) / P;
  const int64_t total = rows * nw;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / nw, wc = idx - r * nw;
    const uint32_t w = in[r * ld32 + wc];
    for (int j = 0; j < P; ++j) {
      const int64_t c = wc * P + j;
      if (c >= cols) break;
      const uint32_t x = (w >> (j * W)) & em;
      if (elem_bytes == 1)
        static_cast<uint8_t*>(X)[r * ldx + c] = (uint8_t)x;
      else
        static_cast<uint16_t*>(X)[r * ldx + c] = (uint16_t)x;
    }
  }
}

int grid_for(int64_t work) {
  const int64_t b = (work + 255) / 256;
  return (int)(b < 1 ? 1 : b > 65535 * 8 ? 65535 * 8 : b);
}

}  // namespace

NjPlan plan_newton_john(int e, int64_t m, int64_t n, int64_t k, bool packed, int num_sms) {
  NjPlan pl{};
  // 32-bit words per row of C: packed rows are written up to their last 64-bit word
  const int64_t nw = packed ? 2 * ceil_div(n, 64 / packed_width(e)) : ceil_div(n, 32 / packed_width(e));
  pl.nw = nw;
  // lanes per row: four words each, up to the whole warp
  int lg = 0;
  while (lg < 5 && (int64_t(4) << lg) < nw) ++lg;
  const int G = 32 >> lg;
  pl.lg = lg;
  pl.tiles_n = ceil_div(nw, int64_t(4) << lg);
  // rows per thread: up to 16 (tiles of 128 rows and more amortise the tables),
  // fewer when the tile would be mostly past the last row
  int R = 16;
  while (R * G > 32) R /= 2;
  while (R > 1 && (int64_t)kWarps * (R / 2) * G >= m) R /= 2;
  // Fill the GPU (two CTAs per SM): split k over a cluster first, then
  // shorten the tiles.
  const int KT = nj_chunk(e);
  const int64_t want = 2 * (int64_t)num_sms;
  int ks = 1;
  int64_t tiles_m = ceil_div(m, (int64_t)kWarps * R * G);
  // Shorter tiles only while the CTAs still fit one wave: a second wave of
  // short-lived CTAs cost more than the longer tiles (GF(4) 4000^2 x 64:
  // 44 against 54 us).
  while (tiles_m * pl.tiles_n * ks < want) {
    if (ks < 8 && ceil_div(k, (int64_t)KT) >= 2 * ks) {
      ks *= 2;
    } else if (R > 1 && ceil_div(m, (int64_t)kWarps * (R / 2) * G) > tiles_m &&
               ceil_div(m, (int64_t)kWarps * (R / 2) * G) * pl.tiles_n * ks <= want) {
      R /= 2;
      tiles_m = ceil_div(m, (int64_t)kWarps * R * G);
    } else {
      break;
    }
  }
  pl.R = R;
  pl.tiles_m = tiles_m;
  pl.ks = ks;
  pl.kper = round_up(ceil_div(k, ks), KT);
  return pl;
}

cudaError_t launch_newton_john(int e, const NjParams& p0, const NjPlan& pl, cudaStream_t s, int64_t* launches) {
  if (p0.m <= 0 || p0.n <= 0 || p0.k <= 0) return cudaSuccess;
  if (pl.tiles_m > 0x7fffffff || pl.tiles_n > 65535 || pl.ks < 1 || pl.ks > 8) return cudaErrorInvalidValue;
  NjParams p = p0;
  p.lg = pl.lg;
  p.ks = pl.ks;
  p.kper = pl.kper;
  p.nw = pl.nw;
  if (launches) ++*launches;
  switch (e) {
    case 2: return nj_launch<2>(p, pl.R, pl.tiles_m, pl.tiles_n, s);
    case 3: return nj_launch<3>(p, pl.R, pl.tiles_m, pl.tiles_n, s);
    case 4: return nj_launch<4>(p, pl.R, pl.tiles_m, pl.tiles_n, s);
    case 5: return nj_launch<5>(p, pl.R, pl.tiles_m, pl.tiles_n, s);
    case 6: return nj_launch<6>(p, pl.R, pl.tiles_m, pl.tiles_n, s);
    case 7: return nj_launch<7>(p, pl.R, pl.tiles_m, pl.tiles_n, s);
    case 8: return nj_launch<8>(p, pl.R, pl.tiles_m, pl.tiles_n, s);
    case 9: return nj_launch<9>(p, pl.R, pl.tiles_m, pl.tiles_n, s);
    case 10: return nj_launch<10>(p, pl.R, pl.tiles_m, pl.tiles_n, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_to_packed(int e, int64_t rows, int64_t cols, const void* X, int64_t ldx, uint32_t* out,
                             int64_t ld32, int* status, cudaStream_t s, int64_t* launches) {
  if (rows <= 0 || ld32 <= 0) return cudaSuccess;
  if (launches) ++*launches;
  to_packed_kernel<<<grid_for(rows * ld32), 256, 0, s>>>(e, rows, cols, X, ldx, e <= 8 ? 1 : 2, out, ld32, status);
  return cudaGetLastError();
}

cudaError_t launch_from_packed(int e, int64_t rows, int64_t cols, const uint32_t* in, int64_t ld32, void* X,
                               int64_t ldx, cudaStream_t s, int64_t* launches) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const int64_t nw = ceil_div(cols, 32 / packed_width(e));
  if (launches) ++*launches;
  from_packed_kernel<<<grid_for(rows * nw), 256, 0, s>>>(e, rows, cols, in, ld32, X, ldx, e <= 8 ? 1 : 2);
  return cudaGetLastError();
}

}  // namespace m4rie
