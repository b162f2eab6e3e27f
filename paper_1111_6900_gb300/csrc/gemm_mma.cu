// GF(2) slice GEMM on the legacy warp-level tensor instructions, in two
// encodings of the same 0/1 operands:
//   - INT8: mma.sync.m16n8k32 s8 x s8 -> s32 on byte planes (0 / 1);
//   - b1:   mma.sync.m16n8k256 b1 x b1 -> s32 with AND + popcount, on the
//           bit planes of the popc form (256 entries of K in 32 bytes).
// Each int32 accumulator holds the exact count sum_t a_t b_t (parity is
// unaffected even by wrap-around, since (x mod 2^32) mod 2 = x mod 2).  Per
// register the two fragment layouts cover the same bytes (a thread's a0 is
// bytes 4 t .. 4 t + 3 of row g of the 32-byte K step, a2 the same 16 bytes
// on), so one kernel body serves both; A's and B's fragments hold the same K
// positions bit for bit, which is all the AND + popcount needs.  sm_103a has
// no tcgen05 kind::i8, and both instructions run far below the tcgen05
// rates; these forms exist to measure those routes.
//
// Layout as for the tcgen05 form (alpha^j-B schedule): A planes [Mp][e*Kp],
// B planes in groups of e*G rows (slice i of element c at row i*G + c).
// Block tile 128 rows x BN plane rows (BN = e*G <= 160), 8 warps as 4 x 2,
// warp tile 32 x BN/2, k-steps of 64 bytes double-buffered with cp.async.
#include "m4rie_internal.cuh"

namespace m4rie {
namespace {

constexpr int BK = 64;        // bytes of K per stage
constexpr int PITCH = BK + 16;  // padded shared row (bytes)
constexpr int MAXBN = 160;

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

template <int NT, bool B1>  // n8 tiles per warp (BN = 16 * NT); B1: the b1 AND-popc instruction
__global__ void __launch_bounds__(256) mma_s8_kernel(const uint8_t* __restrict__ A, const uint8_t* __restrict__ B,
                                                     int64_t ld, const __grid_constant__ TcParams p) {
  constexpr int BN = 16 * NT;
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t* As = smem;                          // [2][128][PITCH]
  uint8_t* Bs = smem + 2 * 128 * PITCH;        // [2][BN][PITCH]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp & 3, wn = warp >> 2;      // warp position: rows 32*wm, plane rows (BN/2)*wn
  const int g = lane >> 2, t4 = lane & 3;
  const int64_t m0 = (int64_t)blockIdx.x * 128;
  const int64_t n0 = (int64_t)blockIdx.y * BN;  // first B plane row of this block
  const int ksteps = (int)((ld + BK - 1) / BK);

  auto load = [&](int ks, int st) {
    const int64_t k0 = (int64_t)ks * BK;
    for (int idx = tid; idx < 128 * 4; idx += 256) {
      const int row = idx >> 2, ch = idx & 3;
      const int64_t k = k0 + ch * 16;
      cp_async16(As + (st * 128 + row) * PITCH + ch * 16, A + (m0 + row) * ld + (k < ld ? k : 0), k < ld);
    }
    for (int idx = tid; idx < BN * 4; idx += 256) {
      const int row = idx >> 2, ch = idx & 3;
      const int64_t k = k0 + ch * 16;
      cp_async16(Bs + (st * BN + row) * PITCH + ch * 16, B + (n0 + row) * ld + (k < ld ? k : 0), k < ld);
    }
  };

  int acc[2][NT][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0;

  load(0, 0);
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (int ks = 0; ks < ksteps; ++ks) {
    if (ks + 1 < ksteps) load(ks + 1, (ks + 1) & 1);
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();
    const uint8_t* as = As + (ks & 1) * 128 * PITCH;
    const uint8_t* bs = Bs + (ks & 1) * BN * PITCH;
#pragma unroll
    for (int kk = 0; kk < BK; kk += 32) {
      uint32_t a[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const uint8_t* r0 = as + (32 * wm + 16 * i + g) * PITCH + kk + 4 * t4;
        const uint8_t* r1 = r0 + 8 * PITCH;
        a[i][0] = *reinterpret_cast<const uint32_t*>(r0);
        a[i][1] = *reinterpret_cast<const uint32_t*>(r1);
        a[i][2] = *reinterpret_cast<const uint32_t*>(r0 + 16);
        a[i][3] = *reinterpret_cast<const uint32_t*>(r1 + 16);
      }
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const uint8_t* rb = bs + ((BN / 2) * wn + 8 * j + g) * PITCH + kk + 4 * t4;
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(rb);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(rb + 16);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          if (B1)
            asm volatile(
                "mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+r"(acc[i][j][0]), "+r"(acc[i][j][1]), "+r"(acc[i][j][2]), "+r"(acc[i][j][3])
                : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b0), "r"(b1));
          else
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+r"(acc[i][j][0]), "+r"(acc[i][j][1]), "+r"(acc[i][j][2]), "+r"(acc[i][j][3])
                : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b0), "r"(b1));
        }
      }
    }
    __syncthreads();
  }

  // Epilogue: parity bits of the 128 x BN tile into shared memory (one bit per
  // (row, plane row)), then field elements: element c of the group has bit i
  // at plane row i*G + c.
  uint32_t* sbits = reinterpret_cast<uint32_t*>(smem);  // [128][BN/32 + 1]
  constexpr int WPR = BN / 32 + 1;
  for (int idx = tid; idx < 128 * WPR; idx += 256) sbits[idx] = 0;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int row = 32 * wm + 16 * i + g + 8 * (h >> 1);
        const int col = (BN / 2) * wn + 8 * j + 2 * t4 + (h & 1);
        if (acc[i][j][h] & 1) atomicOr(&sbits[row * WPR + (col >> 5)], 1u << (col & 31));
      }
  __syncthreads();
  const int G = p.G, E = p.e;
  const int64_t c0 = (int64_t)blockIdx.y * G;
  bool bad = false;
  for (int idx = tid; idx < 128 * G; idx += 256) {
    const int rl = idx / G, cl = idx - rl * G;
    const int64_t r = m0 + rl, c = c0 + cl;
    if (r >= p.m || c >= p.n) continue;
    uint32_t val = 0;
    for (int i = 0; i < E; ++i) {
      const int col = i * G + cl;
      val |= ((sbits[rl * WPR + (col >> 5)] >> (col & 31)) & 1u) << i;
    }
    if (p.elem_bytes == 1) {
      uint8_t* dst = static_cast<uint8_t*>(p.C) + r * p.ldc + c;
      if (p.add) {
        const uint32_t old = *dst;
        bad |= old > p.emask;
        val ^= old & p.emask;
      }
      *dst = (uint8_t)val;
    } else {
      uint16_t* dst = static_cast<uint16_t*>(p.C) + r * p.ldc + c;
      if (p.add) {
        const uint32_t old = *dst;
        bad |= old > p.emask;
        val ^= old & p.emask;
      }
      *dst = (uint16_t)val;
    }
  }
  if (bad) atomicOr(p.status, kStatusRange);
}

template <int NT, bool B1>
cudaError_t run(const uint8_t* A, const uint8_t* B, int64_t ld, const TcParams& p, cudaStream_t s) {
  const size_t smem = (size_t)2 * (128 + 16 * NT) * PITCH;
  cudaError_t err =
      cudaFuncSetAttribute(mma_s8_kernel<NT, B1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  mma_s8_kernel<NT, B1><<<dim3((unsigned)p.tiles_m, (unsigned)p.tiles_n), 256, smem, s>>>(A, B, ld, p);
  return cudaGetLastError();
}

template <bool B1>
cudaError_t dispatch(const uint8_t* a, const uint8_t* b, int64_t ld, const TcParams& p, cudaStream_t s) {
  switch (p.BN / 16) {
    case 1: return run<1, B1>(a, b, ld, p, s);
    case 2: return run<2, B1>(a, b, ld, p, s);
    case 3: return run<3, B1>(a, b, ld, p, s);
    case 4: return run<4, B1>(a, b, ld, p, s);
    case 5: return run<5, B1>(a, b, ld, p, s);
    case 6: return run<6, B1>(a, b, ld, p, s);
    case 7: return run<7, B1>(a, b, ld, p, s);
    case 8: return run<8, B1>(a, b, ld, p, s);
    case 9: return run<9, B1>(a, b, ld, p, s);
    case 10: return run<10, B1>(a, b, ld, p, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int mma_group(int e) {
  int best = 0;
  for (int g = 1; e * g <= MAXBN; ++g)
    if ((e * g) % 16 == 0) best = g;
  return best;
}

cudaError_t launch_mma(bool b1, const void* A, const void* B, int64_t ld, const TcParams& p, cudaStream_t s,
                       int64_t* launches) {
  if (p.tiles_m <= 0 || p.tiles_n <= 0) return cudaSuccess;
  if (p.tiles_n > 65535 || ld % 16 != 0) return cudaErrorInvalidValue;
  if (launches) ++*launches;
  const uint8_t* a = static_cast<const uint8_t*>(A);
  const uint8_t* b = static_cast<const uint8_t*>(B);
  return b1 ? dispatch<true>(a, b, ld, p, s) : dispatch<false>(a, b, ld, p, s);
}

}  // namespace m4rie
