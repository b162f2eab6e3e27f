// Bilinear schedules that reduce one GF(2^e) matrix product to GF(2) products
// (Section 5) and the field arithmetic the host needs to build them.
//
// A schedule is a list of r products P_p = L_p(A) * R_p(B), where L_p and R_p
// are XOR sums of slices (bitmasks over slice indices), and for every output
// slice s a bitmask over p saying which products are XORed into C_s.  The
// reduction modulo f is folded into those output masks.
//
// Karatsuba-like schedules are built recursively from three constructions
// and checked symbolically before use (a bilinear map over GF(2) is fixed by
// its values on the basis pairs (x^i, x^j)):
//   * base cases: 1 product for degree-0 factors, 3 for two coefficients
//     (the GF(4) formula of Section 5), 6 for three coefficients;
//   * splitting a = a_lo + x^h a_hi: lo*lo, hi*hi, (lo+hi)(lo+hi)
//     (2 r(h) + r(n-h) products);
//   * nesting n = u v: an outer schedule over blocks of u coefficients whose
//     block products use an inner schedule (r(u) r(v) products).
//
// Shorter formulas for the field product itself (the product reduced modulo
// f, whose bilinear rank can be below that of the polynomial product) come
// from a flip-graph search (schedules/search.py) and are stored in
// schedule_table.inc, one per e, each written for one field polynomial f_e.
// A formula for f_e serves every irreducible f of degree e through the field
// isomorphism x -> beta, beta a root of f in GF(2)[x]/f_e: with Phi the
// matrix whose column i is beta^i, a *_f b = Phi^-1 (Phi a *_fe Phi b), so
// L' = L Phi, R' = R Phi, W' = Phi^-1 W.  The shorter of the two schedules is
// used, after the same symbolic check on every basis pair.
#include "schedule.h"

#include <algorithm>
#include <map>
#include <utility>

namespace m4rie {

int poly_degree(uint32_t f) {
  int d = -1;
  while (f >> (d + 1)) ++d;
  return d;
}

static uint32_t poly_mod(uint32_t a, uint32_t b) {
  const int db = poly_degree(b);
  while (a && poly_degree(a) >= db) a ^= b << (poly_degree(a) - db);
  return a;
}

bool poly_irreducible(uint32_t f) {
  const int e = poly_degree(f);
  if (e < 1) return false;
  for (uint32_t d = 2; d < (1u << (e / 2 + 1)); ++d) {
    const int dd = poly_degree(d);
    if (dd >= 1 && dd <= e / 2 && poly_mod(f, d) == 0) return false;
  }
  return true;
}

uint32_t x_pow_mod(int e, uint32_t f, int d) {
  uint32_t a = 1;
  for (int i = 0; i < d; ++i) {
    a <<= 1;
    if (a >> e & 1u) a ^= f;
  }
  return a;
}

void alpha_b_masks(int e, uint32_t f, uint16_t* amask, uint16_t* bmask) {
  for (int j = 0; j < e; ++j) amask[j] = (uint16_t)(1u << j);
  // plane (j, i) of B: coefficient i of alpha^j * b = sum_l b_l [x^(j+l) mod f]_i
  for (int i = 0; i < e; ++i)
    for (int j = 0; j < e; ++j) {
      uint32_t m = 0;
      for (int l = 0; l < e; ++l)
        if (x_pow_mod(e, f, j + l) >> i & 1u) m |= 1u << l;
      bmask[i * e + j] = (uint16_t)m;
    }
}

namespace {

struct Bilinear {
  int n = 0;
  std::vector<uint32_t> L, R, W;  // W: bitmask over output coefficients 0 .. 2n-2
  int r() const { return (int)L.size(); }
};

Bilinear base(int n) {
  Bilinear b;
  b.n = n;
  if (n == 1) {
    b.L = {1};
    b.R = {1};
    b.W = {1};
  } else if (n == 2) {
    // a0b0 -> c0 + c1, a1b1 -> c1 + c2, (a0+a1)(b0+b1) -> c1
    b.L = {1, 2, 3};
    b.R = {1, 2, 3};
    b.W = {0x3, 0x6, 0x2};
  } else {
    // three coefficients: a_i b_i (i = 0, 1, 2) and (a_i + a_j)(b_i + b_j)
    b.L = {1, 2, 4, 3, 5, 6};
    b.R = {1, 2, 4, 3, 5, 6};
    b.W = {0x07, 0x0E, 0x1C, 0x02, 0x04, 0x08};
  }
  return b;
}

Bilinear split(const Bilinear& H, const Bilinear& Lo, int h, int l) {
  // a = lo + x^h hi, lo has h coefficients, hi has l <= h
  Bilinear b;
  b.n = h + l;
  const uint32_t lmask = (1u << l) - 1;
  for (int p = 0; p < H.r(); ++p) {  // lo * lo contributes at x^0 and -x^h
    b.L.push_back(H.L[p]);
    b.R.push_back(H.R[p]);
    b.W.push_back(H.W[p] ^ (H.W[p] << h));
  }
  for (int p = 0; p < Lo.r(); ++p) {  // hi * hi contributes at x^2h and -x^h
    b.L.push_back(Lo.L[p] << h);
    b.R.push_back(Lo.R[p] << h);
    b.W.push_back((Lo.W[p] << (2 * h)) ^ (Lo.W[p] << h));
  }
  for (int p = 0; p < H.r(); ++p) {  // (lo + hi)(lo + hi) at x^h
    b.L.push_back(H.L[p] | ((H.L[p] & lmask) << h));
    b.R.push_back(H.R[p] | ((H.R[p] & lmask) << h));
    b.W.push_back(H.W[p] << h);
  }
  return b;
}

Bilinear nest(const Bilinear& In, const Bilinear& Out) {
  // blocks of u = In.n coefficients, v = Out.n blocks
  const int u = In.n;
  Bilinear b;
  b.n = u * Out.n;
  for (int po = 0; po < Out.r(); ++po)
    for (int pi = 0; pi < In.r(); ++pi) {
      uint32_t L = 0, R = 0, W = 0;
      for (int s = 0; s < Out.n; ++s) {
        if (Out.L[po] >> s & 1u) L |= In.L[pi] << (u * s);
        if (Out.R[po] >> s & 1u) R |= In.R[pi] << (u * s);
      }
      for (int d = 0; d < 2 * Out.n - 1; ++d)
        if (Out.W[po] >> d & 1u) W ^= In.W[pi] << (u * d);
      b.L.push_back(L);
      b.R.push_back(R);
      b.W.push_back(W);
    }
  return b;
}

bool verify(const Bilinear& b) {
  for (int i = 0; i < b.n; ++i)
    for (int j = 0; j < b.n; ++j) {
      uint32_t out = 0;
      for (int p = 0; p < b.r(); ++p)
        if ((b.L[p] >> i & 1u) && (b.R[p] >> j & 1u)) out ^= b.W[p];
      if (out != (1u << (i + j))) return false;
    }
  return true;
}

// A field-product formula: r terms (L, R, W) for GF(2)[x]/f, W over the e
// output coefficients.
struct FieldFormula {
  int e;
  uint32_t f;
  int r;
  uint32_t t[3 * 64];
};
const FieldFormula kTable[] = {
#include "schedule_table.inc"
};

// a * b in GF(2)[x]/f (degree e), by shift and add.
uint32_t field_mul(int e, uint32_t f, uint32_t a, uint32_t b) {
  uint32_t r = 0;
  for (int i = e - 1; i >= 0; --i) {
    r <<= 1;
    if (r >> e & 1u) r ^= f;
    if (b >> i & 1u) r ^= a;
  }
  return r;
}

int parity(uint32_t x) { return __builtin_parity(x); }

// Columns of the inverse of the e x e GF(2) matrix with columns col[0..e-1]
// (bit masks); false if it is singular.
bool invert_cols(int e, const uint32_t* col, uint32_t* inv) {
  // row i of [M | I]: bit j = M[i][j] for j < e, bit e + j = I[i][j]
  uint32_t row[16];
  for (int i = 0; i < e; ++i) {
    row[i] = 1u << (e + i);
    for (int j = 0; j < e; ++j)
      if (col[j] >> i & 1u) row[i] |= 1u << j;
  }
  for (int c = 0; c < e; ++c) {
    int piv = -1;
    for (int i = c; i < e && piv < 0; ++i)
      if (row[i] >> c & 1u) piv = i;
    if (piv < 0) return false;
    std::swap(row[c], row[piv]);
    for (int i = 0; i < e; ++i)
      if (i != c && (row[i] >> c & 1u)) row[i] ^= row[c];
  }
  // column j of M^-1: bit i = bit e + j of row i
  for (int j = 0; j < e; ++j) {
    inv[j] = 0;
    for (int i = 0; i < e; ++i)
      if (row[i] >> (e + j) & 1u) inv[j] |= 1u << i;
  }
  return true;
}

// The table's formula for degree e carried over to the field polynomial f;
// false if there is none.
bool field_formula(int e, uint32_t f, Bilinear* out) {
  const FieldFormula* ff = nullptr;
  for (const FieldFormula& x : kTable)
    if (x.e == e) ff = &x;
  if (!ff || ff->r < 1 || ff->r > 64) return false;
  // beta: a root of f in GF(2)[x]/f_e (Horner on f's coefficients)
  uint32_t beta = 0;
  for (uint32_t c = 1; c < (1u << e) && !beta; ++c) {
    uint32_t v = 0;
    for (int d = e; d >= 0; --d) v = field_mul(e, ff->f, v, c) ^ ((f >> d) & 1u);
    if (v == 0) beta = c;
  }
  if (!beta) return false;
  uint32_t phi[16], inv[16];
  phi[0] = 1;
  for (int i = 1; i < e; ++i) phi[i] = field_mul(e, ff->f, phi[i - 1], beta);
  if (!invert_cols(e, phi, inv)) return false;
  out->n = e;
  out->L.clear();
  out->R.clear();
  out->W.clear();
  for (int p = 0; p < ff->r; ++p) {
    uint32_t L = 0, R = 0, W = 0;
    for (int i = 0; i < e; ++i) {
      if (parity(ff->t[3 * p] & phi[i])) L |= 1u << i;
      if (parity(ff->t[3 * p + 1] & phi[i])) R |= 1u << i;
      if (ff->t[3 * p + 2] >> i & 1u) W ^= inv[i];
    }
    out->L.push_back(L);
    out->R.push_back(R);
    out->W.push_back(W);
  }
  return true;
}

const Bilinear& best(int n) {
  static std::map<int, Bilinear> memo;
  auto it = memo.find(n);
  if (it != memo.end()) return it->second;
  Bilinear b;
  if (n <= 3) {
    b = base(n);
  } else {
    bool have = false;
    for (int h = (n + 1) / 2; h < n; ++h) {
      Bilinear c = split(best(h), best(n - h), h, n - h);
      if (!have || c.r() < b.r()) {
        b = c;
        have = true;
      }
    }
    for (int u = 2; u < n; ++u)
      if (n % u == 0) {
        Bilinear c = nest(best(u), best(n / u));
        if (c.r() < b.r()) b = c;
      }
  }
  return memo[n] = b;
}

}  // namespace

bool karatsuba_schedule(int e, uint32_t f, Schedule* out) {
  if (e < 1 || e > 10) return false;
  const Bilinear& b = best(e);
  if (!verify(b) || b.r() > 64) return false;
  Bilinear fb;
  const bool field = field_formula(e, f, &fb) && fb.r() < b.r();
  const Bilinear& use = field ? fb : b;
  out->e = e;
  out->r = use.r();
  out->amask.assign(use.L.begin(), use.L.end());
  out->bmask.assign(use.R.begin(), use.R.end());
  for (int s = 0; s < 10; ++s) out->out_mask[s] = 0;
  // field formula: W_p are output coefficients already; polynomial formula:
  // C_s = sum_d [x^d mod f]_s c_d,  c_d = sum_p [d in W_p] P_p
  for (int p = 0; p < use.r(); ++p) {
    uint32_t red = 0;
    if (field) red = use.W[p];
    else
      for (int d = 0; d < 2 * e - 1; ++d)
        if (use.W[p] >> d & 1u) red ^= x_pow_mod(e, f, d);
    for (int s = 0; s < e; ++s)
      if (red >> s & 1u) out->out_mask[s] |= 1ull << p;
  }
  // end-to-end symbolic check over the field: sum_p [i in L_p][j in R_p] col_p == x^(i+j) mod f
  for (int i = 0; i < e; ++i)
    for (int j = 0; j < e; ++j) {
      uint32_t v = 0;
      for (int p = 0; p < use.r(); ++p)
        if ((use.L[p] >> i & 1u) && (use.R[p] >> j & 1u))
          for (int s = 0; s < e; ++s)
            if (out->out_mask[s] >> p & 1ull) v ^= 1u << s;
      if (v != x_pow_mod(e, f, i + j)) return false;
    }
  return true;
}

}  // namespace m4rie
