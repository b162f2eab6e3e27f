// Internal declarations shared by the translation units of the library.
#pragma once
#include <cstdint>
#include <utility>
#include <cuda_runtime.h>
#include <cuda.h>

namespace m4rie {

// Device status bits (sticky word owned by the context).
enum : int { kStatusRange = 1, kStatusTimeout = 2, kStatusSingular = 4 };

// Programmatic dependent launch.  A kernel launched with the attribute may
// start while the previous kernel of the stream is finishing; pdl_enter()
// waits until that kernel has completed and its writes are visible, then lets
// the next kernel launch early in turn.  Kernels call it before their first
// access to global memory.  Without the attribute both instructions return at
// once.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// cudaLaunchKernelEx with the programmatic-serialization attribute when pdl.
template <typename... Params, typename... Args>
cudaError_t launch_ex(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                      Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Operand plane formats.  Every plane entry is parity(x & mask) for one
// element x and one GF(2)-linear mask, stored as:
enum PlaneFmt : int {
  kFmtBit = 0,   // 1 bit, 32-bit words along K, least significant bit first
  kFmtByte = 1,  // 1 byte per entry: 0 or `one` (0x01 for INT8, 0x38 for FP8 E4M3 1.0)
  kFmtNib = 2,   // 4 bits per entry, two per byte (low nibble first): 0 or `one` (0x2 = E2M1 1.0)
};

constexpr int kMaxMasks = 128;

// Layout of the planes generated from one input matrix (A, or B transposed).
// Mask q = (b * nb + i) * kb + j produces the entries of input row r at
// element offset  b*bstride + orow(r, i)*ld + j*Kp + t, with
//   slice-major:   orow(r, i) = (r / G) * nb * G + i * G + (r % G)
//   element-major: orow(r, i) = (r / G) * nb * G + (r % G) * nb + i   (emajor)
// so a group of nb*G rows holds the nb slices of G consecutive inputs.
struct PackParams {
  const void* X;      // input elements
  int64_t ldx;        // leading dimension of X in elements
  int elem_bytes;     // 1 or 2
  int64_t rows;       // input rows (A: m; B read by columns: n)
  int64_t K;          // inner dimension k
  int64_t rows_p;     // padded rows per batch plane (multiple of G and of the GEMM's M tile)
  int fmt;
  uint32_t one;
  int P, nb, kb, G;
  int64_t Kp;         // padded K per k-block, multiple of 128
  int64_t ld;         // output row length (entries) = kb * Kp
  int64_t bstride;    // entries between batch planes
  uint32_t emask;     // 2^e - 1
  int e;              // number of slice bits of an element
  int vec;            // X and its rows are 16-byte aligned: 128-bit loads allowed
  int emajor;         // element-major row order inside a group (see above)
  void* out;
  int* status;
  uint16_t mask[kMaxMasks];
  // Filled by plane_offsets() (the launchers call it on their copy): byte
  // offset of plane q's row 0, entry 0 from out, and ceil(2^40 / G) so that
  // r / G = (r * gmul) >> 40 for r < 2^31, G < 512.
  int64_t qoff[kMaxMasks];
  uint64_t gmul;
  int pdl;            // launch with programmatic dependent launch
};

// Fill qoff and gmul of p from its layout fields; false if G is out of range.
bool plane_offsets(PackParams& p);

// Pack launchers (pack.cu).  launch_pack_planes: rows of X (rows x K, row
// stride ldx) are the planes' rows.  launch_pack_cols: columns of X (K x rows,
// row stride ldx) are the planes' rows, transposed on the way through shared
// memory.
cudaError_t launch_pack_planes(const PackParams& p, cudaStream_t s, int64_t* launches);
cudaError_t launch_pack_cols(const PackParams& p, cudaStream_t s, int64_t* launches);
// Both at once (A by rows, B by columns) in one launch.
cudaError_t launch_pack_pair(const PackParams& a, const PackParams& b, cudaStream_t s, int64_t* launches);

// Batched forms: job j owns blocks [start[j], start[j+1]) of one launch (all
// jobs of a launch share the element width and the plane format).
int64_t pack_job_blocks(const PackParams& p);
cudaError_t launch_pack_batched(const PackParams* d_jobs, const int64_t* d_start, int njobs, int64_t blocks, int fmt,
                                int elem_bytes, cudaStream_t s, int64_t* launches);

// Column planes of many jobs (X read by columns, no transpose): blocks per job
// and the launch over the job table (same conventions as the row version).
int64_t cols_job_blocks(const PackParams& p);
cudaError_t launch_cols_batched(const PackParams* d_jobs, const int64_t* d_start, int njobs, int64_t blocks, int fmt,
                                int elem_bytes, cudaStream_t s, int64_t* launches);

// Public slice format (Section 3.2): pack.cu.
cudaError_t launch_slice(int e, int64_t rows, int64_t cols, const void* elems, uint64_t* slices,
                         int64_t ld_words, int* status, cudaStream_t s, int64_t* launches);
cudaError_t launch_cling(int e, int64_t rows, int64_t cols, const uint64_t* slices, int64_t ld_words,
                         void* elems, cudaStream_t s, int64_t* launches);

// Karatsuba recombination: out bits from r parity planes (pack.cu).
struct RecombineParams {
  const uint32_t* P;  // r bit planes, plane p row i at P + (p*rows_p + i)*ldw
  int64_t ldw;        // words per parity-plane row
  int64_t rows_p;
  // blocked planes (the tcgen05 GEMM's layout, see TcParams): tiles of tcols
  // columns (a multiple of 16, at most 256) held in the first
  // ceil(tcols / 32) of a block row's 8 words, tiles_n column tiles, bstride
  // words between planes
  int blocked, tcols;
  int64_t tiles_n, bstride;
  int r;
  int e;
  int64_t m, n;
  void* C;
  int64_t ldc;
  int elem_bytes;
  int add;
  uint32_t emask;
  int* status;
  uint64_t out_mask[10];  // bit p of out_mask[s]: product p contributes to output slice s
  int pdl;                // launch with programmatic dependent launch
};
cudaError_t launch_recombine(const RecombineParams& p, cudaStream_t s, int64_t* launches);
// Batched form: job j owns blocks [start[j], start[j + 1]) (all jobs of one
// launch share the element width; e <= 8 for bytes, 9..10 for halfwords).
int64_t recombine_job_blocks(const RecombineParams& p);
cudaError_t launch_recombine_batched(const RecombineParams* d_jobs, const int64_t* d_start, int njobs,
                                     int64_t blocks, int elem_bytes, cudaStream_t s, int64_t* launches);

// ---------------------------------------------------------------- popc form
// Tile constants of the bit-packed GEMM (gemm_popc.cu).
constexpr int kPopcBM = 128;
int popc_group(int e);  // elements per block column (G of the B-side plane layout)

struct PopcParams {
  const uint32_t* A;  // [Mp][ldw]
  const uint32_t* B;  // [groups * e * G][ldw]  (fused)  or  [r][Np][ldw] (parity)
  int64_t ldw;        // words per row
  int64_t m, n;
  int e;
  void* C;            // fused: elements; parity: bit planes
  int64_t ldc;        // fused: elements per row of C; parity: words per plane row
  int elem_bytes;
  int add;
  uint32_t emask;
  int* status;
  // parity (batched) mode
  int batch;
  int64_t a_bstride, b_bstride, c_bstride;  // words between batch planes
  int pdl;            // launch with programmatic dependent launch
};
cudaError_t launch_popc_fused(const PopcParams& p, cudaStream_t s, int64_t* launches);
cudaError_t launch_popc_parity(const PopcParams& p, cudaStream_t s, int64_t* launches);

// ---------------------------------------------------------------- tcgen05 form
constexpr int kTcBM = 128;
int tc_group(int e, int fmt);  // elements per tile column: tile N = e * G

struct TcParams {
  int64_t m, n;
  int e, G, BN;
  int tiles_m, tiles_n;
  int batch;          // independent products (parity mode); 1 otherwise
  int64_t a_brows, b_brows;  // plane rows between products in the A / B tensor maps
  int kblocks;        // K' / 128 bytes
  int kc;             // k-blocks per accumulation chunk (bounds each FP32 count)
  int group_m;        // tile raster: group_m m-tiles per super-column
  void* C;
  int64_t ldc;
  int elem_bytes;
  int add;
  uint32_t emask;
  int* status;
  int mode;           // 0: elements, 2: parity planes, 3: Karatsuba recombined in the epilogue
  // parity mode: the planes are stored in blocks of 128 rows x 8 words (256
  // columns, the tile's BN / 32 <= 8 words and zeros), block (tm, tn) of
  // product b at word b * p_bstride + (tm * tiles_n + tn) * 1024, row i of
  // the block at 8 * i (tiles_n counts column tiles; tm counts 128-row tiles)
  int64_t p_bstride;  // parity mode: words between products
  uint64_t wait_limit_ns;
  const int* tile_job;  // batched launches: job of every global tile
  int f4nv;             // FP4: 1 = kind::mxf4nvf4 (UE4M3 scales per 16), 0 = kind::mxf4 (UE8M0 per 32)
  int stall_test;       // test hook: the epilogue first waits on a barrier that is never signalled
  int cluster;          // 3: 2-SM pairs (tiles_m must be even), 1: single CTAs
  int pdl;              // launch with programmatic dependent launch
  // mode 3 (Karatsuba with the recombination in the epilogue; 2-SM pairs, e <= 8):
  // every product of an output tile runs on one pair, back to back
  uint8_t qmask[64];    // bit s: product b feeds output slice s
  int vec_c;            // C and its rows are 16-byte aligned: 16-byte element stores
};
// fmt: kFmtByte (E4M3) or kFmtNib (E2M1, block scaled).
cudaError_t launch_tc(int fmt, const void* Aplanes, int64_t a_rows, const void* Bplanes, int64_t b_rows,
                      int64_t ld_bytes, const TcParams& p, int num_sms, cudaStream_t s, int64_t* launches);

// One product of a batched persistent launch (element epilogue, alpha^j-B
// layout).  Its tiles are global tiles [tile_start, tile_start + tiles_m *
// tiles_n), m-fastest.  Tensor maps live in device memory with the job.
struct alignas(alignof(CUtensorMap)) TcJob {
  CUtensorMap ma, mb;
  void* C;
  int64_t m, n, ldc;
  int e, G, BN, kblocks, kc, tiles_m, tiles_n, elem_bytes, add;
  uint32_t emask;
  int64_t tile_start;
  // mode 0: alpha^j-B product, elements into C (batch 1); mode 2: batch
  // GF(2) products (Karatsuba), parity planes into C in the blocked layout of
  // TcParams, product b's planes a_brows (b_brows) rows on in the A (B) map
  int mode, batch;
  int64_t a_brows, b_brows, p_bstride;
};
bool tc_make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t ld_bytes, int box_rows);
cudaError_t launch_tc_batched(int fmt, const TcJob* d_jobs, const int* d_tile_job, int njobs, int64_t total_tiles,
                              int* status, uint64_t wait_limit_ns, int num_sms, cudaStream_t s, int64_t* launches);

// ---------------------------------------------------------------- legacy mma.sync forms
int mma_group(int e);  // elements per block column: block N = e * G <= 160
// b1 = false: INT8 (byte planes); b1 = true: b1 AND + popcount (bit planes).
cudaError_t launch_mma(bool b1, const void* Aplanes, const void* Bplanes, int64_t ld_bytes, const TcParams& p,
                       cudaStream_t s, int64_t* launches);

// ---------------------------------------------------------------- helpers
inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
inline int64_t ceil_div(int64_t x, int64_t m) { return (x + m - 1) / m; }

}  // namespace m4rie
