// Bit-packed GF(2) slice GEMM on the CUDA cores ("popc form").
//
// A GF(2) product of bit-packed rows is acc ^= a & b per 32-bit word (one
// LOP3 per 32 bit-multiply-adds), and the GF(2) sum over the inner dimension
// is the parity of the accumulated word, popc(acc) & 1.  With the alpha^j-B
// schedule the whole GF(2^e) product is one such GEMM over the concatenated
// inner dimension (j, t), producing the e output slices of every element
// directly (Section 5: the product reduced to GF(2) products; the reduction mod
// f is folded into the B operand as in the alpha^k B step of Algorithm 2).
//
// Tiling: 256 threads, 128 rows x G elements (e*G plane rows) per block,
// 8 rows x (e * G/16) plane rows per thread, k-tiles of 32 words (1024 bits)
// double-buffered in shared memory with cp.async.  Shared rows are padded to
// 36 words so that 16 consecutive B rows hit distinct bank groups.
#include "m4rie_internal.cuh"

namespace m4rie {
namespace {

constexpr int BKW = 32;     // words per k-tile
constexpr int PITCH = 36;   // shared row pitch in words
constexpr int STAGES = 2;

__device__ __forceinline__ uint32_t andxor(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0x6A;" : "=r"(d) : "r"(a), "r"(b), "r"(c));  // (a & b) ^ c
  return d;
}

__device__ __forceinline__ void cp_async16(uint32_t* dst, const uint32_t* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// E = degree, TNC = elements per thread (G = 16 * TNC elements per block).
template <int E, int TNC, typename OutT>
__global__ void __launch_bounds__(256, 2) popc_fused(const __grid_constant__ PopcParams p) {
  constexpr int G = 16 * TNC;
  constexpr int RB = E * G;
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* As = smem;                               // [STAGES][128][PITCH]
  uint32_t* Bs = smem + STAGES * kPopcBM * PITCH;    // [STAGES][RB][PITCH]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * kPopcBM;
  const int64_t g = blockIdx.y;
  pdl_enter();
  const uint32_t* Ag = p.A + m0 * p.ldw;
  const uint32_t* Bg = p.B + g * RB * p.ldw;
  const int ktiles = (int)((p.ldw + BKW - 1) / BKW);

  auto load = [&](int kt, int st) {
    const int64_t w0 = (int64_t)kt * BKW;
    uint32_t* as = As + st * kPopcBM * PITCH;
    uint32_t* bs = Bs + st * RB * PITCH;
#pragma unroll
    for (int it = 0; it < (kPopcBM * 8) / 256; ++it) {
      const int idx = tid + it * 256, row = idx >> 3, ch = idx & 7;
      const int64_t w = w0 + ch * 4;
      const bool ok = w < p.ldw;
      cp_async16(as + row * PITCH + ch * 4, Ag + row * p.ldw + (ok ? w : 0), ok);
    }
    for (int idx = tid; idx < RB * 8; idx += 256) {
      const int row = idx >> 3, ch = idx & 7;
      const int64_t w = w0 + ch * 4;
      const bool ok = w < p.ldw;
      cp_async16(bs + row * PITCH + ch * 4, Bg + row * p.ldw + (ok ? w : 0), ok);
    }
  };

  uint32_t acc[8][TNC][E];
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int v = 0; v < TNC; ++v)
#pragma unroll
      for (int i = 0; i < E; ++i) acc[q][v][i] = 0;

  load(0, 0);
  cp_commit();
  for (int kt = 0; kt < ktiles; ++kt) {
    if (kt + 1 < ktiles) load(kt + 1, (kt + 1) & 1);
    cp_commit();
    cp_wait<1>();
    __syncthreads();
    const uint32_t* as = As + (kt & 1) * kPopcBM * PITCH + ty * PITCH;
    const uint32_t* bs = Bs + (kt & 1) * RB * PITCH + tx * PITCH;
#pragma unroll 1
    for (int s = 0; s < BKW / 4; ++s) {
      uint4 a[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = *reinterpret_cast<const uint4*>(as + q * 16 * PITCH + 4 * s);
#pragma unroll
      for (int v = 0; v < TNC; ++v)
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const uint4 b = *reinterpret_cast<const uint4*>(bs + (i * G + 16 * v) * PITCH + 4 * s);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            uint32_t t = acc[q][v][i];
            t = andxor(a[q].x, b.x, t);
            t = andxor(a[q].y, b.y, t);
            t = andxor(a[q].z, b.z, t);
            t = andxor(a[q].w, b.w, t);
            acc[q][v][i] = t;
          }
        }
    }
    __syncthreads();
  }

  OutT* C = static_cast<OutT*>(p.C);
  bool bad = false;
  // with accumulation, the old values of 4 row groups are loaded before any
  // of them is written, so the loads' latencies overlap
#pragma unroll
  for (int q0 = 0; q0 < 8; q0 += 4) {
    uint32_t old[4][TNC];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int v = 0; v < TNC; ++v) {
        const int64_t r = m0 + ty + 16 * (q0 + q), c = g * G + tx + 16 * v;
        old[q][v] = p.add && r < p.m && c < p.n ? (uint32_t)C[r * p.ldc + c] : 0u;
      }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t r = m0 + ty + 16 * (q0 + q);
#pragma unroll
      for (int v = 0; v < TNC; ++v) {
        const int64_t c = g * G + tx + 16 * v;
        if (r < p.m && c < p.n) {
          uint32_t val = 0;
#pragma unroll
          for (int i = 0; i < E; ++i) val |= (uint32_t)(__popc(acc[q0 + q][v][i]) & 1) << i;
          if (p.add) {
            bad |= old[q][v] > p.emask;
            val ^= old[q][v] & p.emask;
          }
          C[r * p.ldc + c] = (OutT)val;
        }
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(p.status, kStatusRange);
}

// Parity mode (Karatsuba products): batch of independent GF(2) GEMMs
// P_b = L_b(A) R_b(B); output bit planes, 128 rows x 128 columns per block,
// 8 x 8 per thread.
__global__ void __launch_bounds__(256, 2) popc_parity(const __grid_constant__ PopcParams p) {
  constexpr int RB = 128;
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* As = smem;
  uint32_t* Bs = smem + STAGES * kPopcBM * PITCH;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * kPopcBM;
  const int64_t n0 = (int64_t)blockIdx.y * RB;
  pdl_enter();
  const int b = blockIdx.z;
  const uint32_t* Ag = p.A + b * p.a_bstride + m0 * p.ldw;
  const uint32_t* Bg = p.B + b * p.b_bstride + n0 * p.ldw;
  const int ktiles = (int)((p.ldw + BKW - 1) / BKW);

  auto load = [&](int kt, int st) {
    const int64_t w0 = (int64_t)kt * BKW;
    uint32_t* as = As + st * kPopcBM * PITCH;
    uint32_t* bs = Bs + st * RB * PITCH;
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int idx = tid + it * 256, row = idx >> 3, ch = idx & 7;
      const int64_t w = w0 + ch * 4;
      const bool ok = w < p.ldw;
      cp_async16(as + row * PITCH + ch * 4, Ag + row * p.ldw + (ok ? w : 0), ok);
      cp_async16(bs + row * PITCH + ch * 4, Bg + row * p.ldw + (ok ? w : 0), ok);
    }
  };
  uint32_t acc[8][8];
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[q][v] = 0;
  load(0, 0);
  cp_commit();
  for (int kt = 0; kt < ktiles; ++kt) {
    if (kt + 1 < ktiles) load(kt + 1, (kt + 1) & 1);
    cp_commit();
    cp_wait<1>();
    __syncthreads();
    const uint32_t* as = As + (kt & 1) * kPopcBM * PITCH + ty * PITCH;
    const uint32_t* bs = Bs + (kt & 1) * RB * PITCH + tx * PITCH;
#pragma unroll 1
    for (int s = 0; s < BKW / 4; ++s) {
      uint4 a[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = *reinterpret_cast<const uint4*>(as + q * 16 * PITCH + 4 * s);
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const uint4 bb = *reinterpret_cast<const uint4*>(bs + 16 * v * PITCH + 4 * s);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          uint32_t t = acc[q][v];
          t = andxor(a[q].x, bb.x, t);
          t = andxor(a[q].y, bb.y, t);
          t = andxor(a[q].z, bb.z, t);
          t = andxor(a[q].w, bb.w, t);
          acc[q][v] = t;
        }
      }
    }
    __syncthreads();
  }
  // Output bit (r, c) of plane b: columns of this block are n0 + tx + 16 v.
  // Gather the 128 column bits of each row through shared memory.
  uint32_t* sbits = smem;  // [128 rows][4 words]
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int rl = ty + 16 * q;
    uint32_t part[4] = {0, 0, 0, 0};
#pragma unroll
    for (int v = 0; v < 8; ++v)  // column tx + 16 v is bit tx + 16 (v & 1) of word v >> 1
      part[v >> 1] |= (uint32_t)(__popc(acc[q][v]) & 1) << (tx + 16 * (v & 1));
    // 16 threads (tx) share the row: OR-reduce across the half-warp.
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      uint32_t x = part[w];
      x |= __shfl_xor_sync(0xffffffffu, x, 1);
      x |= __shfl_xor_sync(0xffffffffu, x, 2);
      x |= __shfl_xor_sync(0xffffffffu, x, 4);
      x |= __shfl_xor_sync(0xffffffffu, x, 8);
      part[w] = x;
    }
    if (tx < 4) sbits[rl * 4 + tx] = tx == 0 ? part[0] : tx == 1 ? part[1] : tx == 2 ? part[2] : part[3];
  }
  __syncthreads();
  uint32_t* P = static_cast<uint32_t*>(p.C) + b * p.c_bstride;
  for (int idx = tid; idx < 128 * 4; idx += 256) {
    const int rl = idx >> 2, w = idx & 3;
    P[(m0 + rl) * p.ldc + (n0 >> 5) + w] = sbits[idx];
  }
}

template <int E, int TNC>
cudaError_t run_fused(const PopcParams& p, cudaStream_t s) {
  constexpr int G = 16 * TNC;
  const int64_t gx = ceil_div(p.m, kPopcBM), gy = ceil_div(p.n, G);
  if (gx > 0x7fffffffLL || gy > 65535) return cudaErrorInvalidConfiguration;
  const size_t smem = (size_t)STAGES * (kPopcBM + E * G) * PITCH * 4;
  cudaError_t err;
  if (p.elem_bytes == 2) {
    err = cudaFuncSetAttribute(popc_fused<E, TNC, uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    err = launch_ex(popc_fused<E, TNC, uint16_t>, dim3((unsigned)gx, (unsigned)gy), dim3(256), smem, s, p.pdl != 0, p);
    if (err != cudaSuccess) return err;
  } else {
    err = cudaFuncSetAttribute(popc_fused<E, TNC, uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    err = launch_ex(popc_fused<E, TNC, uint8_t>, dim3((unsigned)gx, (unsigned)gy), dim3(256), smem, s, p.pdl != 0, p);
    if (err != cudaSuccess) return err;
  }
  return cudaGetLastError();
}

}  // namespace

int popc_group(int e) { return e == 2 ? 64 : (e <= 4 ? 32 : 16); }

cudaError_t launch_popc_fused(const PopcParams& p, cudaStream_t s, int64_t* launches) {
  if (p.m <= 0 || p.n <= 0) return cudaSuccess;
  if (launches) ++*launches;
  switch (p.e) {
    case 2: return run_fused<2, 4>(p, s);
    case 3: return run_fused<3, 2>(p, s);
    case 4: return run_fused<4, 2>(p, s);
    case 5: return run_fused<5, 1>(p, s);
    case 6: return run_fused<6, 1>(p, s);
    case 7: return run_fused<7, 1>(p, s);
    case 8: return run_fused<8, 1>(p, s);
    case 9: return run_fused<9, 1>(p, s);
    case 10: return run_fused<10, 1>(p, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_popc_parity(const PopcParams& p, cudaStream_t s, int64_t* launches) {
  if (p.m <= 0 || p.n <= 0 || p.batch <= 0) return cudaSuccess;
  const int64_t gx = ceil_div(p.m, kPopcBM), gy = ceil_div(p.n, 128);
  if (gx > 0x7fffffffLL || gy > 65535 || p.batch > 65535) return cudaErrorInvalidConfiguration;
  const size_t smem = (size_t)STAGES * (kPopcBM + 128) * PITCH * 4;
  cudaError_t err = cudaFuncSetAttribute(popc_parity, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  err = launch_ex(popc_parity, dim3((unsigned)gx, (unsigned)gy, (unsigned)p.batch), dim3(256), smem, s, p.pdl != 0, p);
  if (launches) ++*launches;
  return err != cudaSuccess ? err : cudaGetLastError();
}

}  // namespace m4rie
