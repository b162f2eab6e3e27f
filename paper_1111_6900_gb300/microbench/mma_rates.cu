// tcgen05.mma issue-rate microbenchmark (sm_103a).
//
// One CTA per SM keeps its operands resident in shared memory (zeros: the
// rate does not depend on the values) and issues MMAs back to back from one
// thread into a TMEM accumulator, committing to an mbarrier every 4 MMAs the
// way the GEMM's MMA warp does.  It reports MACs per SM clock and the implied
// whole-GPU rate for the shapes and kinds the slice GEMM uses: kind::f8f6f4
// (E4M3, K = 32), kind::mxf4 (E2M1, scale_vec::2X, K = 64) and kind::mxf4nvf4
// (E2M1, scale_vec::4X, K = 64), M = 128, several N; and the same kinds as
// 2-SM MMAs (cta_group::2, M = 256: each CTA of a 2-CTA cluster holds 128 rows
// of A, half of B and 128 lanes of the accumulator).  Every wait is bounded.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

namespace {

constexpr int SMEM = 160 * 1024;  // also keeps one CTA per SM
constexpr int SF_COL = 496;       // block-scale factors, outside the accumulator
constexpr uint64_t LIMIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// KIND 0: f8f6f4 E4M3; 1: mxf4 (UE8M0 scales); 2: mxf4nvf4 (UE4M3 scales)
template <int KIND>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t sf, uint32_t acc) {
  if (KIND == 0)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else if (KIND == 1)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %5, 0;\n"
        "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%4], p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(sf), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %5, 0;\n"
        "tcgen05.mma.cta_group::1.kind::mxf4nvf4.block_scale.scale_vec::4X [%0], %1, %2, %3, [%4], [%4], p;\n}\n" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc), "r"(sf), "r"(acc)
        : "memory");
}

__host__ __device__ constexpr uint32_t idesc_of(int kind, int M, int N) {
  return kind == 0 ? ((1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24))
                   : ((1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | (kind == 2 ? 0u : (1u << 23)) |
                      ((uint32_t)(M >> 4) << 24));
}

template <int KIND>
__global__ void __launch_bounds__(128, 1) mma_rate(int n, int iters, unsigned long long* cycles, int* status) {
  extern __shared__ uint8_t raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = sm;                 // 128 rows x 128 bytes
  uint8_t* sB = sm + 128 * 128;     // 256 rows x 128 bytes
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + 256 * 128);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2);
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < (128 + 256) * 128 / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bars)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bars + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // zeros visible to the tensor core
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(slot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *slot;
  if (KIND != 0) {
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + SF_COL;
    const uint32_t v = KIND == 2 ? 0x38383838u : 0x7F7F7F7Fu;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(v)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x == 0) {
    const uint32_t idesc = idesc_of(KIND, 128, n);
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB), done = smem_u32(bars), step = smem_u32(bars + 1);
    const long long c0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        mma<KIND>(tmem, sdesc(a0 + 32 * k), sdesc(b0 + 32 * k), idesc, tmem + SF_COL, (it | k) ? 1u : 0u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(step)
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done) : "memory");
    const uint64_t t0 = gtimer();
    bool ok = false;
    while (!(ok = mbar_try(done, 0)) && gtimer() - t0 < LIMIT_NS) {
    }
    cycles[blockIdx.x] = (unsigned long long)(clock64() - c0);
    if (!ok) atomicOr(status, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

template <int KIND>
__device__ __forceinline__ void mma2(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t sf, uint32_t acc) {
  if (KIND == 0)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else if (KIND == 1)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %5, 0;\n"
        "tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%4], p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(sf), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %5, 0;\n"
        "tcgen05.mma.cta_group::2.kind::mxf4nvf4.block_scale.scale_vec::4X [%0], %1, %2, %3, [%4], [%4], p;\n}\n" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc), "r"(sf), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// 2-SM form: launched as clusters of 2 CTAs; the even CTA issues every MMA.
template <int KIND>
__global__ void __launch_bounds__(128, 1) mma_rate_pair(int n, int iters, unsigned long long* cycles, int* status) {
  extern __shared__ uint8_t raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = sm;              // this CTA's 128 rows of A
  uint8_t* sB = sm + 128 * 128;  // this CTA's half of B (<= 128 rows)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + 128 * 128);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2);
  const int warp = threadIdx.x >> 5;
  uint32_t rank;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  for (int i = threadIdx.x; i < 256 * 128 / 16; i += blockDim.x) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bars)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bars + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    // one warp of each CTA of the pair allocates collectively
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(slot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *slot;
  if (KIND != 0) {
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + SF_COL;
    const uint32_t v = KIND == 2 ? 0x38383838u : 0x7F7F7F7Fu;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(v)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync();  // both CTAs: barriers, operands and scale factors ready
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x == 0) {
    const uint32_t done = smem_u32(bars), step = smem_u32(bars + 1);
    const long long c0 = clock64();
    if (rank == 0) {
      const uint32_t idesc = idesc_of(KIND, 256, n);
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          mma2<KIND>(tmem, sdesc(a0 + 32 * k), sdesc(b0 + 32 * k), idesc, tmem + SF_COL, (it | k) ? 1u : 0u);
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                step),
            "h"((uint16_t)3)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
              done),
          "h"((uint16_t)3)
          : "memory");
    }
    const uint64_t t0 = gtimer();
    bool ok = false;
    while (!(ok = mbar_try(done, 0)) && gtimer() - t0 < LIMIT_NS) {
    }
    cycles[blockIdx.x] = (unsigned long long)(clock64() - c0);
    if (!ok) atomicOr(status, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync();  // no CTA frees tensor memory while its peer's MMAs may still run
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

template <int KIND>
int run_pair(const char* name, int n, int sms, int clock_khz) {
  const int iters = 4096;
  const int grid = sms & ~1;
  unsigned long long* d_cyc = nullptr;
  int* d_status = nullptr;
  cudaMalloc(&d_cyc, sizeof(unsigned long long) * grid);
  cudaMalloc(&d_status, sizeof(int));
  cudaMemset(d_status, 0, sizeof(int));
  cudaFuncSetAttribute(mma_rate_pair<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = SMEM;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t err = cudaLaunchKernelEx(&cfg, mma_rate_pair<KIND>, n, iters, d_cyc, d_status);  // warm-up
  cudaEventRecord(e0);
  if (err == cudaSuccess) err = cudaLaunchKernelEx(&cfg, mma_rate_pair<KIND>, n, iters, d_cyc, d_status);
  cudaEventRecord(e1);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  if (err != cudaSuccess) {
    printf("%s pair N=%d: CUDA error %s\n", name, n, cudaGetErrorString(err));
    return 1;
  }
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  std::vector<unsigned long long> cyc(grid);
  int status = 0;
  cudaMemcpy(cyc.data(), d_cyc, sizeof(unsigned long long) * grid, cudaMemcpyDeviceToHost);
  cudaMemcpy(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost);
  unsigned long long cmax = 0;
  for (auto c : cyc) cmax = c > cmax ? c : cmax;
  const int K = KIND == 0 ? 32 : 64;
  const double macs_sm = (double)iters * 4 * 128 * n * K;  // per SM: 128 of the 256 rows
  const double mac_per_clk = macs_sm / (double)cmax;
  printf("%-9s M=256 N=%3d K=%2d (2-SM): %7.0f MAC/clk/SM  -> %6.2f PFLOP/s at %d MHz; %6.2f PFLOP/s by events%s\n",
         name, n, K, mac_per_clk, 2.0 * mac_per_clk * grid * clock_khz * 1e3 / 1e15, clock_khz / 1000,
         2.0 * macs_sm * grid / (ms * 1e-3) / 1e15, status ? "  [TIMEOUT]" : "");
  cudaFree(d_cyc);
  cudaFree(d_status);
  return status;
}

template <int KIND>
int run(const char* name, int n, int sms, int clock_khz) {
  const int iters = 4096;
  unsigned long long* d_cyc = nullptr;
  int* d_status = nullptr;
  cudaMalloc(&d_cyc, sizeof(unsigned long long) * sms);
  cudaMalloc(&d_status, sizeof(int));
  cudaMemset(d_status, 0, sizeof(int));
  cudaFuncSetAttribute(mma_rate<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  mma_rate<KIND><<<sms, 128, SMEM>>>(n, iters, d_cyc, d_status);  // warm-up
  cudaEventRecord(e0);
  mma_rate<KIND><<<sms, 128, SMEM>>>(n, iters, d_cyc, d_status);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  if (err != cudaSuccess) {
    printf("%s N=%d: CUDA error %s\n", name, n, cudaGetErrorString(err));
    return 1;
  }
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  std::vector<unsigned long long> cyc(sms);
  int status = 0;
  cudaMemcpy(cyc.data(), d_cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost);
  cudaMemcpy(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost);
  unsigned long long cmax = 0;
  for (auto c : cyc) cmax = c > cmax ? c : cmax;
  const int K = KIND == 0 ? 32 : 64;
  const double macs_cta = (double)iters * 4 * 128 * n * K;
  const double mac_per_clk = macs_cta / (double)cmax;
  printf("%-9s M=128 N=%3d K=%2d: %7.0f MAC/clk/SM  -> %6.2f PFLOP/s at %d MHz; %6.2f PFLOP/s by events%s\n", name, n,
         K, mac_per_clk, 2.0 * mac_per_clk * sms * clock_khz * 1e3 / 1e15, clock_khz / 1000,
         2.0 * macs_cta * sms / (ms * 1e-3) / 1e15, status ? "  [TIMEOUT]" : "");
  cudaFree(d_cyc);
  cudaFree(d_status);
  return status;
}

}  // namespace

int main() {
  int dev = 0, sms = 0, clock_khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev);
  int bad = 0;
  for (int n : {128, 224, 256}) bad |= run<0>("f8f6f4", n, sms, clock_khz);
  for (int n : {128, 224, 240, 256}) bad |= run<1>("mxf4", n, sms, clock_khz);
  for (int n : {128, 224, 256}) bad |= run<2>("mxf4nvf4", n, sms, clock_khz);
  for (int n : {128, 256}) bad |= run_pair<0>("f8f6f4", n, sms, clock_khz);
  for (int n : {128, 224, 256}) bad |= run_pair<1>("mxf4", n, sms, clock_khz);
  for (int n : {128, 224, 256}) bad |= run_pair<2>("mxf4nvf4", n, sms, clock_khz);
  return bad;
}
