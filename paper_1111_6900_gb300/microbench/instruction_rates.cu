// Instruction-rate microbenchmarks (register-only loops, no memory traffic in the loop).
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e_), __LINE__); return 1; } } while (0)

__global__ void k_lop3(uint32_t* out, int iters, uint32_t seed) {
  uint32_t a[8], b[4], acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = seed * (threadIdx.x + 7 * i + 1);
#pragma unroll
  for (int j = 0; j < 4; ++j) b[j] = seed ^ (threadIdx.x * 13 + j);
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint32_t r;
        asm volatile("lop3.b32 %0, %1, %2, %3, 0x6A;" : "=r"(r) : "r"(a[i]), "r"(b[j]), "r"(acc[i][j]));
        acc[i][j] = r;
      }
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = __funnelshift_l(b[j], b[j], 1);
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s += __popc(acc[i][j]);
  if (s == seed) out[0] = s;
}

__global__ void k_mma_s8(int* out, int iters, uint32_t seed) {
  uint32_t a0 = seed * threadIdx.x, a1 = a0 ^ 1, a2 = a0 ^ 2, a3 = a0 ^ 3, b0 = seed + threadIdx.x, b1 = b0 ^ 5;
  int c[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                   : "+r"(c[i][0]), "+r"(c[i][1]), "+r"(c[i][2]), "+r"(c[i][3])
                   : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  int s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  if (s == (int)seed) out[0] = s;
}

__global__ void k_mma_b1(int* out, int iters, uint32_t seed) {
  uint32_t a0 = seed * threadIdx.x, a1 = a0 ^ 1, a2 = a0 ^ 2, a3 = a0 ^ 3, b0 = seed + threadIdx.x, b1 = b0 ^ 5;
  int c[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      asm volatile("mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                   : "+r"(c[i][0]), "+r"(c[i][1]), "+r"(c[i][2]), "+r"(c[i][3])
                   : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  int s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  if (s == (int)seed) out[0] = s;
}

__global__ void k_mma_f16(float* out, int iters, uint32_t seed) {
  uint32_t a0 = 0x3C003C00u, a1 = a0, a2 = a0, a3 = a0, b0 = 0x3C003C00u, b1 = b0;
  float c[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0.f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                   : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
                   : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  float s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  if (s == (float)seed) out[0] = s;
}

template <typename F>
float timeit(F f) {
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  f(); cudaDeviceSynchronize();
  cudaEventRecord(a); f(); cudaEventRecord(b); cudaEventSynchronize(b);
  float ms; cudaEventElapsedTime(&ms, a, b); return ms;
}

int main() {
  int dev = 0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, dev));
  int clk = 0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  printf("device %s sms %d cc %d.%d clock_khz %d\n", p.name, p.multiProcessorCount, p.major, p.minor, clk);
  void* out; CK(cudaMalloc(&out, 1024));
  int sms = p.multiProcessorCount;
  for (int bpsm : {4, 8}) {
    int blocks = sms * bpsm, threads = 256, iters = 4096;
    float ms = timeit([&] { k_lop3<<<blocks, threads>>>((uint32_t*)out, iters, 12345u); });
    double ops = double(blocks) * threads * iters * 32;
    printf("LOP3 bpsm=%d: %.3f ms, %.3f Tlane-op/s, %.1f lane-op/clk/SM(at %d MHz), bitMAC/s=%.3e\n", bpsm, ms, ops / ms / 1e9,
           ops / (ms * 1e-3) / sms / (clk * 1e3), clk / 1000, ops * 32 / (ms * 1e-3));
  }
  CK(cudaGetLastError());
  for (int bpsm : {4, 8}) {
    int blocks = sms * bpsm, threads = 256, iters = 1024;
    double warps = double(blocks) * threads / 32;
    float ms = timeit([&] { k_mma_s8<<<blocks, threads>>>((int*)out, iters, 7u); });
    double macs = warps * iters * 8 * 16 * 8 * 32;
    printf("MMA s8 m16n8k32 bpsm=%d: %.3f ms, %.3f TOPS (2*MAC)\n", bpsm, ms, 2 * macs / ms / 1e9);
    ms = timeit([&] { k_mma_b1<<<blocks, threads>>>((int*)out, iters, 7u); });
    macs = warps * iters * 8 * 16 * 8 * 256;
    printf("MMA b1 m16n8k256 and.popc bpsm=%d: %.3f ms, %.3f T bitMAC/s\n", bpsm, ms, macs / ms / 1e9);
    ms = timeit([&] { k_mma_f16<<<blocks, threads>>>((float*)out, iters, 7u); });
    macs = warps * iters * 8 * 16 * 8 * 16;
    printf("MMA f16 m16n8k16 bpsm=%d: %.3f ms, %.3f TFLOPS\n", bpsm, ms, 2 * macs / ms / 1e9);
  }
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  return 0;
}
