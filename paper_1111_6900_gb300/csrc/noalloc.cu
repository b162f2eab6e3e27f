// m4rie_mul_noalloc: the bit-packed (popc) alpha^j-B product with its operand
// planes in a fixed, statically allocated device array instead of a
// context-owned workspace, so that the call itself never allocates.
//
// Who needs it: callers that may not allocate device memory on their path.
// Examples are a host framework whose own allocator has already reserved the
// device memory, so that a cudaMalloc from this library would fail or fragment
// its pool; code whose memory footprint must be fixed when the library is
// loaded; and latency-critical loops where cudaMalloc/cudaFree, which can
// synchronise the device, are not acceptable.  Such callers still own and pass
// their inputs and outputs; only the library's scratch comes from here.
//
// The scratch array costs kScratchBytes of device memory on every GPU on
// which the library is loaded, for the life of the process.  Every call shares
// it, so calls whose GPU work overlaps (two streams, two host threads) race on
// it and must be serialised by the caller.  The array keeps the previous
// call's contents: each call's pack kernel rewrites every plane word that its
// GEMM reads, padding included, so nothing is cleared.  The operand planes of
// A are packed by rows and those of B by columns in one launch (B's columns
// are transposed through shared memory on the way), as in the context path.
//
// The array's device address is looked up once per device and cached for the
// life of the process; after cudaDeviceReset the cached address is stale, so
// this entry point must not be called on a device that has been reset.
#include <mutex>

#include "../../include/m4rie_gpu.h"
#include "m4rie_internal.cuh"
#include "schedule.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // operand planes + one status word
constexpr size_t kStatusSlot = kScratchBytes - 256;  // fallback status word when the caller passes none

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device.  In host code the name
// g_scratch is only a host-side stand-in, so the address is fetched once per
// device with cudaGetSymbolAddress (with that device current) and cached.
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, g_scratch);
    if (err != cudaSuccess) return err;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" m4rie_status m4rie_mul_noalloc(int e, uint32_t f, int64_t m, int64_t n, int64_t k, const void* A,
                                          const void* B, void* C, int accumulate, int* device_status,
                                          void* stream_ptr) {
  using namespace m4rie;
  m4rie_status st = m4rie_validate(e, f, m, n, k, A, B, C);
  if (st != M4RIE_OK) return st;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
  const int eb = e <= 8 ? 1 : 2;
  if (m == 0 || n == 0) return M4RIE_OK;
  if (k == 0) {
    if (accumulate) return M4RIE_OK;
    return cudaMemsetAsync(C, 0, (size_t)(m * n) * eb, stream) == cudaSuccess ? M4RIE_OK : M4RIE_ERR_CUDA;
  }
  // Plane sizes of the popc alpha^j-B layout (same as the context path).
  const int G = popc_group(e);
  const int64_t Kp = round_up(k, 128);
  const int64_t ld = (int64_t)e * Kp;  // bits per plane row
  const int64_t Mp = round_up(m, 128);
  const int64_t groups = ceil_div(n, G);
  const int64_t brows = groups * e * G;
  const double a_bytes_d = (double)Mp * ld / 8, b_bytes_d = (double)brows * ld / 8;
  if (a_bytes_d + b_bytes_d + 2048.0 > (double)kStatusSlot) return M4RIE_ERR_SCRATCH;
  const size_t a_bytes = (size_t)round_up(Mp * ld / 8, 1024);
  const size_t b_bytes = (size_t)round_up(brows * ld / 8, 1024);

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return M4RIE_ERR_CUDA;
  void* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return M4RIE_ERR_CUDA;
  uint8_t* Ap = static_cast<uint8_t*>(base);
  uint8_t* Bp = Ap + a_bytes;
  int* status = device_status ? device_status : reinterpret_cast<int*>(static_cast<uint8_t*>(base) + kStatusSlot);

  uint16_t amask[10], bmask[100];
  alpha_b_masks(e, f, amask, bmask);
  PackParams pa{};
  pa.X = A;
  pa.ldx = k;
  pa.elem_bytes = eb;
  pa.rows = m;
  pa.K = k;
  pa.rows_p = Mp;
  pa.fmt = kFmtBit;
  pa.one = 1;
  pa.P = e;
  pa.nb = 1;
  pa.kb = e;
  pa.G = 1;
  pa.Kp = Kp;
  pa.ld = ld;
  pa.emask = (1u << e) - 1;
  pa.e = e;
  pa.vec = (reinterpret_cast<uintptr_t>(A) & 15u) == 0 && (k * eb) % 16 == 0;
  pa.out = Ap;
  pa.status = status;
  for (int j = 0; j < e; ++j) pa.mask[j] = amask[j];
  PackParams pb = pa;  // columns of B (k x n) are the planes' rows
  pb.X = B;
  pb.ldx = n;
  pb.rows = n;
  pb.rows_p = groups * G;
  pb.P = e * e;
  pb.nb = e;
  pb.kb = e;
  pb.G = G;
  pb.out = Bp;
  for (int q = 0; q < e * e; ++q) pb.mask[q] = bmask[q];
  if (launch_pack_pair(pa, pb, stream, nullptr) != cudaSuccess) return M4RIE_ERR_CUDA;

  PopcParams pp{};
  pp.A = reinterpret_cast<const uint32_t*>(Ap);
  pp.B = reinterpret_cast<const uint32_t*>(Bp);
  pp.ldw = ld / 32;
  pp.m = m;
  pp.n = n;
  pp.e = e;
  pp.C = C;
  pp.ldc = n;
  pp.elem_bytes = eb;
  pp.add = accumulate ? 1 : 0;
  pp.emask = (1u << e) - 1;
  pp.status = status;
  if (launch_popc_fused(pp, stream, nullptr) != cudaSuccess) return M4RIE_ERR_CUDA;
  return M4RIE_OK;
}
