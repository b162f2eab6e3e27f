/*
 * m4rie_gpu.h -- C ABI of the GB300 (sm_103a) library for dense matrix
 * multiplication over GF(2^e), 2 <= e <= 10, in the bitsliced form.
 *
 * Method (Section 5, "Karatsuba multiplication"): a matrix over GF(2^e) is a
 * polynomial with GF(2)-matrix coefficients, its slices (Section 3.2).  The
 * product A*B is computed from GF(2) products of slices (or of XOR sums of
 * slices), whose results are recombined and reduced modulo the field
 * polynomial f.  Every result is exact: each call produces the same bits as
 * the plain definition C[r][c] = sum_t A[r][t] * B[t][c] (Algorithm 1).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Field elements (Section 2): the integer sum_i a_i 2^i stands for
 *    sum_i a_i x^i in F2[x]/<f>.  Element arrays are uint8 when e <= 8 and
 *    little-endian uint16 when e is 9 or 10.  Addition is XOR.
 *  - f: bitmask of the field polynomial including the x^e term (for example
 *    0x13 = x^4 + x + 1).  It must have degree exactly e and be irreducible;
 *    primitivity is not required.
 *  - Matrices: contiguous row-major, A is m x k, B is k x n, C is m x n
 *    (leading dimensions k, n, n).
 *  - Pointers: device pointers owned by the caller, unless the name says host.
 *    The library never frees them.  A pointer may be NULL only when the
 *    matrix it points to has no entries.
 *  - Asynchrony: calls enqueue work on the context's stream and return
 *    without waiting.  The return value reports host-side validation and
 *    launch errors only.  Errors found on the device (an entry >= 2^e, a
 *    wait that timed out) set a sticky device status word that
 *    m4rie_get_device_status() reads.  An out-of-range entry is then used
 *    through its low e bits, so the output stays deterministic.
 *  - Zero sizes: m == 0 or n == 0 is a no-op.  k == 0 makes m4rie_mul write
 *    zeros to C and leaves C unchanged for m4rie_addmul.
 *  - Errors never trap or abort on the device.
 *
 * Environment variables read by m4rie_create (tuning and measurement):
 *  - M4RIE_TUNE_CACHE: autotuner cache file to load (see m4rie_tune_load).
 *  - M4RIE_TC_CHUNK: entries per FP32 accumulation chunk of the tcgen05 forms
 *    (at most 2^21, so that every count stays below 2^23).
 *  - M4RIE_TC_CLUSTER: tcgen05 tiles on 2-SM pairs (3, default) or on single
 *    CTAs (1).
 *  - M4RIE_F4_KIND=nvf4: FP4 products with kind::mxf4nvf4 instead of kind::mxf4.
 *  - M4RIE_PDL=0: launch kernels without programmatic dependent launch.
 *  - M4RIE_FUSE_RECOMBINE=1: Karatsuba on 2-SM pairs (e <= 8) recombines in the
 *    GEMM's epilogue instead of a separate kernel (slower on the measured
 *    shapes; off by default).
 *  - M4RIE_ZERO_COPY=0: m4rie_mul_host always stages through device memory.
 */
#ifndef M4RIE_GPU_H
#define M4RIE_GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum m4rie_status {
    M4RIE_OK = 0,
    M4RIE_ERR_ARG = 1,        /* invalid argument: e outside [2,10], negative size, NULL data, bad option */
    M4RIE_ERR_POLY = 2,       /* f does not have degree e or is reducible over GF(2) */
    M4RIE_ERR_ALIAS = 3,      /* the output overlaps an input */
    M4RIE_ERR_RANGE = 4,      /* device: an input entry was >= 2^e (its low e bits were used) */
    M4RIE_ERR_NOMEM = 5,      /* workspace allocation failed */
    M4RIE_ERR_CUDA = 6,       /* a CUDA runtime or driver call failed (see m4rie_last_error) */
    M4RIE_ERR_TIMEOUT = 7,    /* device: a bounded wait inside a kernel ran out; that kernel's output is incomplete */
    M4RIE_ERR_UNSUPPORTED = 8, /* the requested form is not available for this problem or device */
    M4RIE_ERR_SCRATCH = 9,     /* m4rie_mul_noalloc: the operand planes exceed its fixed scratch array */
    M4RIE_ERR_SINGULAR = 10    /* device: a triangular solve met a zero on the diagonal; its output is undefined */
} m4rie_status;

/* How the GF(2) slice products are computed. */
typedef enum m4rie_form {
    M4RIE_FORM_AUTO = 0,   /* autotuned choice (the fastest form measured for this shape class) */
    M4RIE_FORM_POPC = 1,   /* bit-packed slices, AND/XOR on the CUDA cores, parity by popcount */
    M4RIE_FORM_TC_F8 = 2,  /* tcgen05 tensor cores; 0/1 operands encoded exactly as FP8 E4M3, FP32 counts */
    M4RIE_FORM_MMA_S8 = 3, /* legacy warp-level INT8 tensor instructions (mma.sync s8), int32 counts */
    M4RIE_FORM_TC_F4 = 4,  /* tcgen05 block-scaled FP4 (E2M1 0/1 operands, unit scales), FP32 counts */
    M4RIE_FORM_MMA_B1 = 5, /* legacy warp-level binary tensor instructions (mma.sync b1, AND + popcount)
                              on the bit-packed slices, int32 counts */
    M4RIE_FORM_NEWTON_JOHN = 6 /* no slicing: Newton-John tables (Section 4, Algorithms 2 and 3) of the
                              packed rows of B (Section 3.1) in shared memory, one table row added per
                              entry of A; for small products and thin inner dimensions (see
                              m4rie_mul_packed).  Element rows of B and C that start on 16-byte
                              boundaries (base and row stride) move as 16-byte vectors, the fast case */
} m4rie_form;

/* Which bilinear schedule reduces the GF(2^e) product to GF(2) products. */
typedef enum m4rie_schedule {
    M4RIE_SCHED_AUTO = 0,      /* autotuned choice */
    M4RIE_SCHED_ALPHA_B = 1,   /* e^2 products C_i = sum_j A_j (alpha^j B)_i: the schoolbook count,
                                  with the reduction mod f folded into B (Algorithm 2's alpha^k B) */
    M4RIE_SCHED_KARATSUBA = 2  /* Karatsuba-like: fewer products (Table 3), recombined after parity */
} m4rie_schedule;

typedef struct m4rie_ctx m4rie_ctx;

/* One product of a batch (m4rie_mul_batched).  Host-side descriptor; the
 * pointers inside are device pointers. */
typedef struct m4rie_problem {
    int32_t e;
    uint32_t f;
    int64_t m, n, k;
    const void *A;  /* m x k */
    const void *B;  /* k x n */
    void *C;        /* m x n */
    int32_t accumulate; /* 0: C = A B, 1: C += A B */
    int32_t reserved;
} m4rie_problem;

/* Create a context bound to the current CUDA device and to `stream` (a
 * cudaStream_t; NULL means the legacy default stream).  The context owns a
 * device workspace that grows on demand, the device status word and the
 * autotuning cache.  One context per stream; a context is not thread-safe.
 * Returns M4RIE_ERR_ARG if ctx is NULL, M4RIE_ERR_CUDA if no device. */
m4rie_status m4rie_create(m4rie_ctx **ctx, void *stream);

/* Wait for the context's stream, then free everything it owns. */
void m4rie_destroy(m4rie_ctx *ctx);

/* Select the form and the schedule used by later calls (AUTO by default).
 * M4RIE_ERR_ARG for an unknown value. */
m4rie_status m4rie_set_form(m4rie_ctx *ctx, int form);
m4rie_status m4rie_set_schedule(m4rie_ctx *ctx, int schedule);

/* C = A * B over GF(2^e) = F2[x]/<f> (Section 5; result as in Algorithm 1).
 * A: m x k, B: k x n, C: m x n, device pointers, element width from e.
 * C must not overlap A or B (M4RIE_ERR_ALIAS).  Asynchronous on the stream. */
m4rie_status m4rie_mul(m4rie_ctx *ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k,
                       const void *A, const void *B, void *C);

/* C = C + A * B over GF(2^e) (addition is XOR, Section 3.1).  C is read and
 * updated in place; otherwise as m4rie_mul. */
m4rie_status m4rie_addmul(m4rie_ctx *ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k,
                          const void *A, const void *B, void *C);

/* C = A * B (accumulate == 0) or C = C + A * B (accumulate != 0) over
 * GF(2^e) on strided windows (the matrix windows Section 3 takes over from
 * M4RI): row r of A starts at A + r * lda elements, of B at B + r * ldb, of C
 * at C + r * ldc.  Requires lda >= k, ldb >= n, ldc >= n (M4RIE_ERR_ARG);
 * the bytes C spans must not overlap those A or B span (M4RIE_ERR_ALIAS).
 * Otherwise as m4rie_mul; m4rie_mul is m4rie_gemm with lda = k, ldb = ldc = n. */
m4rie_status m4rie_gemm(m4rie_ctx *ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k,
                        const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc,
                        int accumulate);

/* Triangular solving with matrices (Section 4.3, Algorithm 5): B <- T^{-1} * B
 * over GF(2^e), in place.  T is m x m (row stride ldt >= m), upper triangular
 * for m4rie_trsm_upper_left, lower triangular for m4rie_trsm_lower_left; the
 * other triangle is never read, so T may share storage with other data (an
 * in-place PLE, for instance).  B is m x n (row stride ldb >= n) and must not
 * overlap T (M4RIE_ERR_ALIAS).  Blocked and recursive: diagonal blocks of 128
 * rows are inverted in shared memory, every other step is a slice GEMM
 * (m4rie_gemm).  A zero diagonal entry sets the sticky device status
 * M4RIE_ERR_SINGULAR (B is then undefined); an entry >= 2^e sets
 * M4RIE_ERR_RANGE.  Asynchronous on the context's stream; uses a context-owned
 * scratch of ceil(m / 128) x 128 x 128 elements.  The first solve on given
 * operands and settings is also recorded as a CUDA graph, which later solves
 * with the same pointers, sizes, field and settings replay (reading the
 * buffers' current contents). */
m4rie_status m4rie_trsm_upper_left(m4rie_ctx *ctx, int e, uint32_t f, int64_t m, int64_t n, const void *T,
                                   int64_t ldt, void *B, int64_t ldb);
m4rie_status m4rie_trsm_lower_left(m4rie_ctx *ctx, int e, uint32_t f, int64_t m, int64_t n, const void *T,
                                   int64_t ldt, void *B, int64_t ldb);

/* Reduced row echelon form over GF(2^e) in place (Section 4.1, Algorithm 4;
 * Section 6): A is m x n with row stride lda >= n.  On return A holds the
 * unique reduced row echelon form of the input, *rank (if rank != NULL) its
 * rank r, and pivots[0 .. r) (if pivots != NULL; room for min(m, n) entries)
 * the pivot column of each of the first r rows.  Runs by panels of 64
 * columns: a candidate block is reduced in shared memory to find the pivots,
 * and the rest of the matrix is updated with slice GEMMs.  Synchronous (it
 * reads the pivot list back for every panel).  Entries >= 2^e set the sticky
 * M4RIE_ERR_RANGE status.  Uses a context-owned scratch of about
 * 64 m + 256 n elements. */
m4rie_status m4rie_echelonize(m4rie_ctx *ctx, int e, uint32_t f, int64_t m, int64_t n, void *A, int64_t lda,
                              int64_t *rank, int64_t *pivots);

/* PLE decomposition over GF(2^e) in place (Section 4.2, in the library's
 * variant of the definition): A = P L E with P a permutation, L (m x r) lower
 * trapezoidal holding the pivots on its diagonal and E (r x n) in row echelon
 * form with leading entries 1.  Pivoting is Algorithm 4's (Section 4.1): for
 * every column the first row at or below the current rank with a non-zero
 * entry is swapped up, so the result is the one that algorithm with Section
 * 4.2's changes gives.  A is m x n with row stride lda >= n.  On return, for
 * rank r:
 *   A[i][t] = L[i][t] for t <= min(i, r - 1);
 *   for k < r: E[k][j] = 0 for j < Q[k], 1 for j = Q[k] (not stored),
 *   A[k][j] for j > Q[k];
 *   every other entry of A is 0.
 * *rank (if rank != NULL) receives r; P (if not NULL, m entries) the swap
 * partners: at step t rows t and P[t] were exchanged (P[t] >= t; P[i] = i for
 * i >= r), so A is recovered from L E by swapping rows t and P[t] for
 * t = r-1 down to 0; Q (if not NULL, n entries) the pivot column of step t
 * in Q[t] for t < r (increasing) and Q[j] = j for j >= r.  P and Q are host
 * arrays.  Runs by panels of 64 columns; synchronous (it reads each panel's
 * pivot list back).  Entries >= 2^e set the sticky M4RIE_ERR_RANGE status.
 * Uses the context-owned scratch of m4rie_echelonize (about 64 m + 256 n
 * elements). */
m4rie_status m4rie_ple(m4rie_ctx *ctx, int e, uint32_t f, int64_t m, int64_t n, void *A, int64_t lda, int64_t *rank,
                       int64_t *P, int64_t *Q);

/* m4rie_mul / m4rie_addmul (accumulate != 0) on HOST buffers: copies A, B
 * (and C when accumulating) to context-owned device memory, computes, copies
 * C back and waits for the stream.  Host buffers may be pageable or pinned.
 * When all three are pinned and mapped into the device's address space and
 * the product moves at most 8 MiB, the kernels read and write them in place
 * instead (no staging copies).  Products of more than 32 MiB with m >= 1024
 * run in four row panels of A and C on two further streams, so that copies
 * of some panels overlap the products of others (B is copied and sliced
 * once). */
m4rie_status m4rie_mul_host(m4rie_ctx *ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k,
                            const void *hostA, const void *hostB, void *hostC, int accumulate);

/* Slicing (Section 3.2, Figure 1): elements (rows x cols, row-major) to e
 * GF(2) slices.  Slice i holds coefficient i of every entry; slice i, row r
 * starts at slices + (i * rows + r) * ld_words; column c is bit (c mod 64) of
 * word floor(c / 64), least significant bit first.  ld_words >= ceil(cols/64);
 * padding bits are written as zero.  Device pointers. */
m4rie_status m4rie_pack(m4rie_ctx *ctx, int e, int64_t rows, int64_t cols, const void *elems,
                        uint64_t *slices, int64_t ld_words);

/* Clinging (Section 3.2): the inverse of m4rie_pack.  Padding bits are ignored. */
m4rie_status m4rie_unpack(m4rie_ctx *ctx, int e, int64_t rows, int64_t cols, const uint64_t *slices,
                          int64_t ld_words, void *elems);

/* Packed representation (Section 3.1, Figure 1): every element padded to
 * m4rie_packed_width(e) bits (2 for e = 2, 4 for e = 3, 4, 8 for e = 5 .. 8,
 * 16 for e = 9, 10: the next length dividing 64), rows of 64-bit words with
 * column c in field (c mod (64 / w)) of word floor(c / (64 / w)), lowest
 * field first.  Returns 0 for e outside [2, 10]. */
int m4rie_packed_width(int e);

/* Elements (rows x cols, row stride lde >= cols elements) to packed rows
 * (row r at words + r * ld_words, ld_words >= ceil(cols / (64 / w))).
 * Padding fields, the bits above e of each field and padding words are written
 * as zero; entries >= 2^e set the sticky M4RIE_ERR_RANGE status.  The two
 * arrays must not overlap (M4RIE_ERR_ALIAS).  Device pointers, asynchronous. */
m4rie_status m4rie_to_packed(m4rie_ctx *ctx, int e, int64_t rows, int64_t cols, const void *elems, int64_t lde,
                             uint64_t *words, int64_t ld_words);

/* The inverse of m4rie_to_packed: reads the low e bits of the first cols
 * fields of every row (padding is ignored) and writes rows x cols elements
 * with row stride lde.  Device pointers, asynchronous. */
m4rie_status m4rie_from_packed(m4rie_ctx *ctx, int e, int64_t rows, int64_t cols, const uint64_t *words,
                               int64_t ld_words, void *elems, int64_t lde);

/* C = A * B (accumulate == 0) or C = C + A * B on packed matrices by
 * Newton-John multiplication (Section 4, Algorithms 2 and 3): for every row t
 * of B a table of its 2^e multiples (for e >= 6 two tables, of the multiples
 * of B_t by scalars of b = ceil(e / 2) bits and of alpha^b B_t by scalars of
 * e - b bits, two lookups per entry) is built in shared memory from the rows
 * alpha^i B_t, and every row r of C adds the table row(s) indexed by A[r][t].
 * A is m x k, B k x n, C m x n, each a packed matrix with row stride lda / ldb
 * / ldc 64-bit words (>= the words of one row).
 * Input padding is ignored; C's padding fields are written as zero.  A field
 * whose bits above e are set sets the sticky M4RIE_ERR_RANGE status (its low
 * e bits are used).  C must not overlap A or B (M4RIE_ERR_ALIAS).  One launch;
 * small products split k over a cluster of up to 8 CTAs and reduce their
 * partial tiles in distributed shared memory.  Asynchronous. */
m4rie_status m4rie_mul_packed(m4rie_ctx *ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k,
                              const uint64_t *A, int64_t lda, const uint64_t *B, int64_t ldb, uint64_t *C,
                              int64_t ldc, int accumulate);

/* Many independent products (each with its own e, f, m, n, k and
 * accumulate flag) in one persistent launch.  `problems` is a HOST array of
 * `count` descriptors (reserved fields zero), validated like m4rie_mul; no
 * output may overlap another output or any input (M4RIE_ERR_ALIAS).
 * With the AUTO, TC_F4 or TC_F8 form the products use the alpha^j-B schedule
 * on the tcgen05 tensor cores: one batched operand-plane kernel per side (the
 * B operands read by columns) and one persistent GEMM over the tiles of all
 * products.
 * That work is recorded once into a CUDA graph, cached in the context with
 * its own device memory, and replayed while the same descriptor array contents
 * are passed (a different array rebuilds it; the first call synchronises the
 * stream).  With the POPC, MMA_S8, MMA_B1 or NEWTON_JOHN form the products run
 * one by one. */
m4rie_status m4rie_mul_batched(m4rie_ctx *ctx, int count, const m4rie_problem *problems);

/* Wait for the stream, return the sticky device status and clear it:
 * M4RIE_OK, or the most severe condition seen since the last call
 * (M4RIE_ERR_TIMEOUT before M4RIE_ERR_SINGULAR before M4RIE_ERR_RANGE). */
m4rie_status m4rie_get_device_status(m4rie_ctx *ctx);

/* Number of GF(2) slice products that `schedule` uses for GF(2^e) with the
 * field polynomial f (e^2 for ALPHA_B).  Negative m4rie_status on error. */
int m4rie_schedule_products(int e, uint32_t f, int schedule);

/* The host-side checks of m4rie_mul on these arguments, without a context,
 * a device or a launch: M4RIE_OK, M4RIE_ERR_ARG, M4RIE_ERR_POLY or
 * M4RIE_ERR_ALIAS.  Pointers are only compared, never dereferenced. */
m4rie_status m4rie_validate(int e, uint32_t f, int64_t m, int64_t n, int64_t k, const void *A, const void *B,
                            const void *C);

/* The masks of a schedule, for inspection: product p multiplies the XOR sum
 * of the A slices in amask[p] by the XOR sum of the B slices in bmask[p];
 * output slice s is the XOR of the products p with bit p of out_mask[s].  For
 * ALPHA_B, product p = i*e + j is A_j times (alpha^j B)_i: amask[p] = 1 << j
 * and bmask[p] holds the coefficients of alpha^j B that make slice i;
 * product p feeds output slice p / e (out_mask is filled only when e*e <= 64).
 * Arrays must hold `cap` entries (out_mask: 10).  Returns the number of
 * products, or a negative m4rie_status. */
int m4rie_schedule_masks(int e, uint32_t f, int schedule, int cap, uint16_t *amask, uint16_t *bmask,
                         uint64_t *out_mask);

/* Autotuner: run every form x schedule x tile raster on synthetic inputs of
 * shape (e, m, n, k) (device memory is allocated for the run and freed), drop
 * any candidate whose output differs from the first candidate's, time the
 * rest with CUDA events on the context's stream, and make the fastest the
 * AUTO choice for the shape class (e, floor(log2(m*n*k))).  Synchronous.
 * The context's explicit form and schedule settings are left unchanged. */
m4rie_status m4rie_tune(m4rie_ctx *ctx, int e, uint32_t f, int64_t m, int64_t n, int64_t k);

/* Autotuner for batched products (m4rie_mul_batched; not in the paper, which
 * multiplies one pair at a time): for every class (e, floor(log2(m n k))) of
 * the given batch, up to 32 of its products (the same shapes, synthetic
 * elements in scratch buffers this call allocates and frees; the batch's own
 * A, B and C are not read or written) run in the persistent batched launch
 * under the alpha^j-B and the Karatsuba-like schedule (Section 5), each
 * recorded, warmed up and timed over five CUDA-graph replays on the context's
 * stream; the faster schedule is kept for that class.  Later m4rie_mul_batched
 * calls take the measured schedule per product; untuned classes keep the
 * rule (Karatsuba for e >= 3).  m4rie_tune_save / m4rie_tune_load keep these
 * choices too.  Synchronises the context's stream.  M4RIE_ERR_UNSUPPORTED if
 * the context's form is not AUTO, TC_F4 or TC_F8 (the batched launch runs on
 * tcgen05 only); argument errors as for m4rie_mul_batched. */
m4rie_status m4rie_tune_batched(m4rie_ctx *ctx, int count, const m4rie_problem *problems);

/* The autotuned choice for the shape class of (e, m, n, k): form and
 * schedule (0 when the class was not tuned) and its measured milliseconds. */
m4rie_status m4rie_tuned_choice(m4rie_ctx *ctx, int e, int64_t m, int64_t n, int64_t k, int *form, int *schedule,
                                double *ms);

/* Save / load the tuned choices as a text file (one line per shape class).
 * m4rie_create loads the file named by the environment variable
 * M4RIE_TUNE_CACHE when it exists. */
m4rie_status m4rie_tune_save(m4rie_ctx *ctx, const char *path);
m4rie_status m4rie_tune_load(m4rie_ctx *ctx, const char *path);

/* Form that AUTO picks for this shape (after m4rie_tune, the measured best). */
int m4rie_resolve_form(m4rie_ctx *ctx, int e, int64_t m, int64_t n, int64_t k);

/* Static description of a status code. */
const char *m4rie_status_string(m4rie_status s);

/* Text of the last CUDA error seen by this context ("" if none). */
const char *m4rie_last_error(m4rie_ctx *ctx);

/* Number of this library's kernels launched through ctx since creation. */
int64_t m4rie_kernel_launches(m4rie_ctx *ctx);

/* Per-phase device timing for measurement.  When enabled, the context
 * records CUDA events on its stream around each phase of every product:
 * operand slicing (pack kernels), the GF(2) slice GEMM, and the
 * recombination / output phase when it is a separate kernel.
 * m4rie_phase_times waits for the stream and returns the accumulated
 * milliseconds and the number of products timed since the last reset
 * (reset = 1 clears them).  Timing adds no synchronisation while enabled. */
m4rie_status m4rie_enable_timing(m4rie_ctx *ctx, int on);
m4rie_status m4rie_phase_times(m4rie_ctx *ctx, double *pack_ms, double *gemm_ms, double *recombine_ms,
                               int64_t *products, int reset);

/* Test hook: limit, in nanoseconds, of every bounded wait inside this
 * context's persistent kernels (default 4e9).  A small value makes those
 * waits run out; the kernel then sets M4RIE_ERR_TIMEOUT and returns. */
m4rie_status m4rie_set_wait_limit_ns(m4rie_ctx *ctx, uint64_t ns);

/* C = A*B (accumulate == 0) or C += A*B (accumulate != 0) over GF(2^e), like
 * m4rie_mul / m4rie_addmul, for callers that may not allocate device memory:
 * for example a host framework whose own allocator has already reserved the
 * GPU's memory, code whose memory footprint must be fixed when the library is
 * loaded, or a latency-critical loop in which cudaMalloc / cudaFree (which can
 * synchronise the device) are not acceptable.  The paper has no counterpart;
 * this is a deployment variant of the bit-packed popc form with the alpha^j-B
 * schedule.
 *
 * No context is needed and the call allocates nothing.  Its operand planes
 * live in one statically allocated device array of 64 MiB that every GPU
 * loading this library holds until the process exits.  Problems whose planes
 * do not fit (Mp*e*Kp/8 + ceil(n/G)*G*e*e*Kp/8 bytes, each rounded up to
 * 1 KiB, plus 2 KiB, above 64 MiB - 256 bytes, with Kp = k rounded up to 128,
 * Mp = m rounded up to 128, G = 64, 32 or 16 for e = 2, 3-4, 5-10; a
 * 4096 x 4096 x 4096 product over GF(2^4) fits) are rejected with
 * M4RIE_ERR_SCRATCH before anything is launched.
 *
 * A, B, C: device pointers as for m4rie_mul.  device_status: optional device
 * int that receives the status bits (1: an entry was >= 2^e, 2: a wait timed
 * out) OR-ed in; with NULL they go to a word inside the scratch array that is
 * never read, so they are lost (the product is computed all the same).  stream: cudaStream_t (NULL = legacy
 * default stream).  Asynchronous like m4rie_mul.
 *
 * The first call on each device looks up the device address of the scratch
 * array (cudaGetSymbolAddress) and caches it for the life of the process;
 * make that first call before any stream capture on that device, and do not
 * call this entry point on a device after cudaDeviceReset (the cached address
 * is then stale).  All calls share the scratch array, which keeps the
 * previous call's contents (each call rewrites every word it reads), so calls
 * whose GPU work overlaps race on it: serialise them. */
m4rie_status m4rie_mul_noalloc(int e, uint32_t f, int64_t m, int64_t n, int64_t k, const void *A, const void *B,
                               void *C, int accumulate, int *device_status, void *stream);

/* Test hook for failure detection: flags & 1 makes every later tcgen05 GEMM
 * launch of this context first wait on a barrier that nothing signals, so that
 * its bounded wait runs out (after the m4rie_set_wait_limit_ns limit), the
 * kernel sets M4RIE_ERR_TIMEOUT, stops and returns; its output is then
 * incomplete.  flags = 0 restores normal operation.  M4RIE_ERR_ARG for
 * unknown flags. */
m4rie_status m4rie_set_test_hook(m4rie_ctx *ctx, int flags);

#ifdef __cplusplus
}
#endif
#endif /* M4RIE_GPU_H */
