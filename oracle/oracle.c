/*
 * CPU oracle for dense matrix multiplication and triangular solving over
 * GF(2^e), 2 <= e <= 10.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA path: no slicing schedule, no precomputed multiples, no tables.
 *
 * Every function is the plain definition it cites, written for clarity and
 * not for speed:
 *
 *   - Field elements (Section 2, "Notation"): GF(2^e) = F2[x]/<f>, deg f = e,
 *     an element sum_i a_i x^i is identified with the integer sum_i a_i 2^i.
 *     f is passed as an integer bitmask that includes the x^e term.
 *   - Field product: polynomial (carry-less) product of the two
 *     representatives, then reduction modulo f.
 *   - Matrix product (Algorithm 1, "Cubic matrix multiplication"): for every
 *     row r of A and every index t of the inner dimension, row t of B is
 *     scaled by A[r][t] and added into row r of C.  The printed loop indices
 *     of Algorithm 1 are garbled; the standard reading C[r][c] =
 *     sum_t A[r][t] * B[t][c] (A is m x l, B is l x n) is used.
 *   - Addition in characteristic 2 is XOR (Section 1 and Section 3.1).
 *   - Field inverse: a^(2^e - 2), since the multiplicative group has order
 *     2^e - 1.
 *   - Triangular solving with matrices (Section 4.3, Algorithm 5): for U
 *     upper triangular, rows of B from the last to the first are scaled by
 *     the inverse diagonal entry and eliminated from the rows above; the
 *     lower-triangular case runs the same steps from the first row down.
 *   - Reduced row echelon form (Section 4.1, Algorithm 4): column by column,
 *     the first row at or below the current rank with a non-zero entry is
 *     scaled to a leading 1, swapped up, and its multiples are added to every
 *     other row to clear the column.
 *   - PLE decomposition (Section 4.2, the library's variant of the
 *     definition): Algorithm 4 with the changes Section 4.2 lists, that is
 *     the swap partners and pivot columns recorded, only the rows below the
 *     pivot cleared and from the column after the pivot on (the multipliers
 *     stay in place as L), and L's columns moved next to the diagonal at the
 *     end by column swaps on and below the diagonal.
 *   - Packed representation (Section 3.1 and Figure 1): each element is
 *     padded to the next field width that divides 64 (2, 4, 8 or 16 bits;
 *     F_32 elements take 8 bits, Figure 1's F_8 elements 4) and a row is a
 *     sequence of 64-bit words, column c in field (c mod (64 / w)) of word
 *     floor(c / (64 / w)), the lowest field first; padding is zero.
 *   - Slicing (Section 3.2 and Figure 1): slice i of a matrix holds
 *     coefficient i (bit i of the integer encoding) of every entry.  Slices
 *     are stored as rows of 64-bit words, column c at bit (c mod 64) of word
 *     floor(c / 64) (least significant bit first), padding bits zero.
 *
 * Parity of every function here is pinned by the tests in tests/ against
 * values fixed independently of this file (Figure 1, the GF(4) example of
 * Section 5, brute-force field axioms, logarithm tables, invariants, and for
 * the solver U * X = B checked with the separately pinned product).
 */
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Section 2: product in F2[x]/<f>.  Carry-less multiply, then reduce the
 * terms of degree 2e-2 down to e by subtracting (XOR) shifted copies of f. */
uint32_t oracle_gf_mul(int e, uint32_t f, uint32_t a, uint32_t b)
{
    uint32_t p = 0;
    for (int i = 0; i < e; i++)
        if ((b >> i) & 1u)
            p ^= a << i;
    for (int d = 2 * e - 2; d >= e; d--)
        if ((p >> d) & 1u)
            p ^= f << (d - e);
    return p;
}

/* Full 2^e x 2^e product table built entry by entry from oracle_gf_mul
 * (used by the tests to compare against independently built tables). */
void oracle_gf_mul_table(int e, uint32_t f, uint16_t *out)
{
    uint32_t q = 1u << e;
    for (uint32_t a = 0; a < q; a++)
        for (uint32_t b = 0; b < q; b++)
            out[(size_t)a * q + b] = (uint16_t)oracle_gf_mul(e, f, a, b);
}

static int oracle_threads = 0;

/* Number of OpenMP threads the matrix routines use (0 = OpenMP default). */
void oracle_set_threads(int n) { oracle_threads = n; }

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return oracle_threads > 0 ? oracle_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/* Algorithm 1: C <- C + A * B when accumulate != 0, C <- A * B otherwise.
 * A is m x k, B is k x n, C is m x n, all row-major with leading dimensions
 * k, n and n, entries stored as uint16 integers < 2^e.  Rows of C are
 * independent, so they are distributed over threads; the per-row work is the
 * algorithm's own loop order (scale row t of B by A[r][t], add to row r). */
void oracle_matmul(int e, uint32_t f, int64_t m, int64_t n, int64_t k,
                   const uint16_t *A, const uint16_t *B, uint16_t *C,
                   int accumulate)
{
    int nt = oracle_get_threads();
    (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t r = 0; r < m; r++) {
        uint16_t *crow = C + r * n;
        if (!accumulate)
            for (int64_t c = 0; c < n; c++)
                crow[c] = 0;
        for (int64_t t = 0; t < k; t++) {
            uint32_t a = A[r * k + t];
            const uint16_t *brow = B + t * n;
            for (int64_t c = 0; c < n; c++)
                crow[c] ^= (uint16_t)oracle_gf_mul(e, f, a, brow[c]);
        }
    }
}

/* Section 3.2 / Figure 1: slicing.  elems is rows x cols (uint16, row-major);
 * slices receives e planes, plane i at slices + i * rows * ld_words, row r of
 * plane i at + r * ld_words; bit (c mod 64) of word floor(c/64) is bit i of
 * elems[r][c].  Padding bits (c >= cols) are written as zero. */
void oracle_slice(int e, int64_t rows, int64_t cols, const uint16_t *elems,
                  uint64_t *slices, int64_t ld_words)
{
    for (int i = 0; i < e; i++) {
        uint64_t *plane = slices + (int64_t)i * rows * ld_words;
        for (int64_t r = 0; r < rows; r++) {
            uint64_t *row = plane + r * ld_words;
            for (int64_t w = 0; w < ld_words; w++)
                row[w] = 0;
            for (int64_t c = 0; c < cols; c++)
                if ((elems[r * cols + c] >> i) & 1u)
                    row[c / 64] |= (uint64_t)1 << (c % 64);
        }
    }
}

/* Section 3.1: bits per element in the packed representation, the smallest
 * of 2, 4, 8, 16 (lengths dividing 64) that holds e bits. */
int oracle_packed_width(int e)
{
    int w = 2;
    while (w < e)
        w *= 2;
    return w;
}

/* Section 3.1 / Figure 1: packed representation.  elems is rows x cols
 * (uint16, row-major); row r of the output starts at words + r * ld_words;
 * element c sits in bits [w * (c mod (64/w)), w * (c mod (64/w)) + w) of word
 * floor(c / (64/w)), w = oracle_packed_width(e).  Everything else is zero. */
void oracle_pack(int e, int64_t rows, int64_t cols, const uint16_t *elems, uint64_t *words,
                 int64_t ld_words)
{
    const int w = oracle_packed_width(e);
    const int per = 64 / w;
    for (int64_t r = 0; r < rows; r++) {
        uint64_t *row = words + r * ld_words;
        for (int64_t j = 0; j < ld_words; j++)
            row[j] = 0;
        for (int64_t c = 0; c < cols; c++)
            row[c / per] |= (uint64_t)elems[r * cols + c] << (w * (c % per));
    }
}

/* Section 3.1: the inverse of oracle_pack.  Padding is ignored: only the low
 * e bits of each field and the first cols fields of a row are read. */
void oracle_unpack(int e, int64_t rows, int64_t cols, const uint64_t *words, int64_t ld_words,
                   uint16_t *elems)
{
    const int w = oracle_packed_width(e);
    const int per = 64 / w;
    for (int64_t r = 0; r < rows; r++)
        for (int64_t c = 0; c < cols; c++) {
            const uint64_t word = words[r * ld_words + c / per];
            elems[r * cols + c] = (uint16_t)((word >> (w * (c % per))) & ((1u << e) - 1u));
        }
}

/* Section 3.2: clinging, the inverse of slicing.  Padding bits are ignored. */
void oracle_cling(int e, int64_t rows, int64_t cols, const uint64_t *slices,
                  int64_t ld_words, uint16_t *elems)
{
    for (int64_t r = 0; r < rows; r++)
        for (int64_t c = 0; c < cols; c++) {
            uint32_t v = 0;
            for (int i = 0; i < e; i++) {
                const uint64_t *row = slices + (int64_t)i * rows * ld_words + r * ld_words;
                v |= (uint32_t)((row[c / 64] >> (c % 64)) & 1u) << i;
            }
            elems[r * cols + c] = (uint16_t)v;
        }
}

/* Field inverse: a^(2^e - 2) by square-and-multiply with oracle_gf_mul (the
 * group of non-zero elements has order 2^e - 1).  Returns 0 for a = 0. */
uint32_t oracle_gf_inv(int e, uint32_t f, uint32_t a)
{
    uint32_t r = 1, base = a, x = (1u << e) - 2;
    if (a == 0)
        return 0;
    while (x) {
        if (x & 1u)
            r = oracle_gf_mul(e, f, r, base);
        base = oracle_gf_mul(e, f, base, base);
        x >>= 1;
    }
    return r;
}

/* Section 4.3, Algorithm 5 (TRSM upper left): B <- U^{-1} * B, U m x m upper
 * triangular (row-major, leading dimension m), B m x n (leading dimension n).
 * For i from m-1 down to 0: row i of B is multiplied by U[i][i]^{-1}, then
 * U[j][i] times row i is added to row j for every j < i.  The algorithm's
 * table T of the multiples of row i is a speed device only; the products
 * U[j][i] * B[i][c] are formed directly.  The row updates for one i are
 * independent and run on several threads.  Returns 0, or -1 if a diagonal
 * entry is zero (no solution is defined; B is left partly updated). */
int oracle_trsm_upper_left(int e, uint32_t f, int64_t m, int64_t n, const uint16_t *U, uint16_t *B)
{
    int nt = oracle_get_threads();
    (void)nt;
    for (int64_t i = m - 1; i >= 0; i--) {
        uint32_t d = U[i * m + i];
        if (d == 0)
            return -1;
        uint32_t dinv = oracle_gf_inv(e, f, d);
        uint16_t *bi = B + i * n;
        for (int64_t c = 0; c < n; c++)
            bi[c] = (uint16_t)oracle_gf_mul(e, f, dinv, bi[c]);
#pragma omp parallel for schedule(static) num_threads(nt) if (i * n > 65536)
        for (int64_t j = 0; j < i; j++) {
            uint32_t x = U[j * m + i];
            uint16_t *bj = B + j * n;
            for (int64_t c = 0; c < n; c++)
                bj[c] ^= (uint16_t)oracle_gf_mul(e, f, x, bi[c]);
        }
    }
    return 0;
}

/* The lower-left counterpart: B <- L^{-1} * B, L m x m lower triangular.  For
 * i from 0 up to m-1: row i is multiplied by L[i][i]^{-1}, then L[j][i] times
 * row i is added to row j for every j > i.  Returns 0, or -1 on a zero
 * diagonal entry. */
int oracle_trsm_lower_left(int e, uint32_t f, int64_t m, int64_t n, const uint16_t *L, uint16_t *B)
{
    int nt = oracle_get_threads();
    (void)nt;
    for (int64_t i = 0; i < m; i++) {
        uint32_t d = L[i * m + i];
        if (d == 0)
            return -1;
        uint32_t dinv = oracle_gf_inv(e, f, d);
        uint16_t *bi = B + i * n;
        for (int64_t c = 0; c < n; c++)
            bi[c] = (uint16_t)oracle_gf_mul(e, f, dinv, bi[c]);
#pragma omp parallel for schedule(static) num_threads(nt) if ((m - i) * n > 65536)
        for (int64_t j = i + 1; j < m; j++) {
            uint32_t x = L[j * m + i];
            uint16_t *bj = B + j * n;
            for (int64_t c = 0; c < n; c++)
                bj[c] ^= (uint16_t)oracle_gf_mul(e, f, x, bi[c]);
        }
    }
    return 0;
}

/* Section 4.1, Algorithm 4: A (m x n, row-major, leading dimension n) is
 * brought to reduced row echelon form in place; returns the rank r.  If
 * pivots is not NULL, pivots[i] receives the pivot column of row i < r.  For
 * every column j: the first row i >= r with A[i][j] != 0 is multiplied by
 * A[i][j]^{-1}, swapped with row r, and A[k][j] times it is added to every
 * other row k; then r grows by one.  (The algorithm's table of the multiples
 * of row r is a speed device; the products are formed directly.  The clearing
 * of the other rows is independent per row and runs on several threads.) */
int64_t oracle_echelon(int e, uint32_t f, int64_t m, int64_t n, uint16_t *A, int64_t *pivots)
{
    int nt = oracle_get_threads();
    (void)nt;
    int64_t r = 0;
    for (int64_t j = 0; j < n && r < m; j++) {
        int64_t i = r;
        while (i < m && A[i * n + j] == 0)
            i++;
        if (i == m)
            continue;
        uint32_t inv = oracle_gf_inv(e, f, A[i * n + j]);
        uint16_t *ai = A + i * n;
        for (int64_t c = 0; c < n; c++)
            ai[c] = (uint16_t)oracle_gf_mul(e, f, inv, ai[c]);
        if (i != r) {
            uint16_t *ar = A + r * n;
            for (int64_t c = 0; c < n; c++) {
                uint16_t t = ar[c];
                ar[c] = ai[c];
                ai[c] = t;
            }
        }
        const uint16_t *pr = A + r * n;
#pragma omp parallel for schedule(static) num_threads(nt) if (m * (n - j) > 65536)
        for (int64_t k = 0; k < m; k++) {
            if (k == r)
                continue;
            uint32_t x = A[k * n + j];
            if (x == 0)
                continue;
            uint16_t *ak = A + k * n;
            for (int64_t c = j; c < n; c++)
                ak[c] ^= (uint16_t)oracle_gf_mul(e, f, x, pr[c]);
        }
        if (pivots)
            pivots[r] = j;
        r++;
    }
    return r;
}

/* Section 4.2, PLE decomposition in the library's variant: A = P L E with P a
 * permutation, L (m x r) lower trapezoidal whose diagonal holds the pivots,
 * and E (r x n) in row echelon form with leading entries 1.  A (m x n,
 * row-major, leading dimension n) is overwritten in place; returns r.
 *
 * For every column j, as in Algorithm 4: the first row i >= r with
 * A[i][j] != 0 is swapped with row r (whole rows), P[r] = i, Q[r] = j.  The
 * entries of row r right of column j are multiplied by A[r][j]^{-1}, so that
 * row r from column j + 1 on is E's row r; A[r][j] stays as L's diagonal
 * entry.  Every row k > r with x = A[k][j] gets x times row r added from
 * column j + 1 on; x stays at (k, j) as L[k][r].  Rows above r are not
 * touched.  Then r grows by one.  At the end L's column t, held in column
 * Q[t], is moved to column t: for t = 0 .. r-1 the columns t and Q[t] are
 * swapped in rows t .. m-1.
 *
 * Result: A[i][t] = L[i][t] for t <= min(i, r - 1); for k < r, E[k][j] = 0
 * for j < Q[k], 1 for j = Q[k] and A[k][j] for j > Q[k]; every other entry
 * of A is 0.  P[i] = i for i >= r and Q[j] = j for j >= r (P has m entries,
 * Q n).  A is recovered from L E by swapping rows t and P[t] for
 * t = r-1 down to 0. */
int64_t oracle_ple(int e, uint32_t f, int64_t m, int64_t n, uint16_t *A, int64_t *P, int64_t *Q)
{
    int nt = oracle_get_threads();
    (void)nt;
    for (int64_t i = 0; i < m; i++)
        P[i] = i;
    for (int64_t j = 0; j < n; j++)
        Q[j] = j;
    int64_t r = 0;
    for (int64_t j = 0; j < n && r < m; j++) {
        int64_t i = r;
        while (i < m && A[i * n + j] == 0)
            i++;
        if (i == m)
            continue;
        if (i != r) {
            uint16_t *ai = A + i * n, *ar = A + r * n;
            for (int64_t c = 0; c < n; c++) {
                uint16_t t = ar[c];
                ar[c] = ai[c];
                ai[c] = t;
            }
        }
        P[r] = i;
        Q[r] = j;
        uint16_t *pr = A + r * n;
        uint32_t inv = oracle_gf_inv(e, f, pr[j]);
        for (int64_t c = j + 1; c < n; c++)
            pr[c] = (uint16_t)oracle_gf_mul(e, f, inv, pr[c]);
#pragma omp parallel for schedule(static) num_threads(nt) if ((m - r) * (n - j) > 65536)
        for (int64_t k = r + 1; k < m; k++) {
            uint32_t x = A[k * n + j];
            if (x == 0)
                continue;
            uint16_t *ak = A + k * n;
            for (int64_t c = j + 1; c < n; c++)
                ak[c] ^= (uint16_t)oracle_gf_mul(e, f, x, pr[c]);
        }
        r++;
    }
    for (int64_t t = 0; t < r; t++) {
        int64_t q = Q[t];
        if (q == t)
            continue;
        for (int64_t k = t; k < m; k++) {
            uint16_t v = A[k * n + t];
            A[k * n + t] = A[k * n + q];
            A[k * n + q] = v;
        }
    }
    return r;
}
