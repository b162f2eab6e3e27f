/* Random walk on the flip graph of rank-one decompositions of a bilinear map
 * over GF(2) (the method of Kauers and Moosbauer, "Flip graphs for matrix
 * multiplication", 2022, restated here for 3-tensors of small size).
 *
 * A scheme is a list of terms (a, b, c): bitmasks over the two input spaces
 * and the output space; it computes the bilinear map T when
 *   sum over terms of [bit i of a][bit j of b] * c  ==  T[i][j]  for all i, j.
 * Moves that keep a scheme correct:
 *   flip       two terms sharing one factor x: (x, y1, z1), (x, y2, z2) become
 *              (x, y1 + y2, z1), (x, y2, z2 + z1);
 *   reduction  two terms sharing two factors merge into one (the third factors
 *              add); a term with a zero factor is dropped;
 *   plus       two terms become three (see plus() below), which opens new
 *              flips.
 * The walk flips at random and reduces whenever it can; after a long plateau
 * it restarts from the best scheme found so far, half of the time with a plus
 * move.
 *
 * Input (stdin): n1 n2 n3 target_rank max_steps plateau seed, the n1*n2 target words
 * T[i][j] (row-major, bit s = output coordinate s), then the starting scheme:
 * r and r lines "a b c".  Output: the best scheme found, in the same form.
 * Every scheme printed is checked against T first. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define RMAX 96

typedef struct {
  uint32_t f[3];
} Term;

static int n1, n2, n3;
static uint32_t T[16][16];

static uint64_t rng_state;
static uint64_t rnd(void) { /* xorshift64* */
  rng_state ^= rng_state >> 12;
  rng_state ^= rng_state << 25;
  rng_state ^= rng_state >> 27;
  return rng_state * 2685821657736338717ull;
}
static int rndn(int n) { return (int)((rnd() >> 33) % (uint64_t)n); }

static int check(const Term* t, int r) {
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n2; ++j) {
      uint32_t acc = 0;
      for (int p = 0; p < r; ++p)
        if ((t[p].f[0] >> i & 1u) && (t[p].f[1] >> j & 1u)) acc ^= t[p].f[2];
      if (acc != T[i][j]) return 0;
    }
  return 1;
}

static void drop(Term* t, int* r, int i) {
  t[i] = t[*r - 1];
  --*r;
}

/* Merge every pair of terms that shares two factors; drop zero terms. */
static void reduce_all(Term* t, int* r) {
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int i = 0; i < *r && !changed; ++i) {
      if (!t[i].f[0] || !t[i].f[1] || !t[i].f[2]) {
        drop(t, r, i);
        changed = 1;
        break;
      }
      for (int j = i + 1; j < *r && !changed; ++j)
        for (int p = 0; p < 3; ++p) {
          const int q = (p + 1) % 3, s = (p + 2) % 3;
          if (t[i].f[q] == t[j].f[q] && t[i].f[s] == t[j].f[s]) {
            t[i].f[p] ^= t[j].f[p];
            drop(t, r, j);
            changed = 1;
            break;
          }
        }
    }
  }
}

/* One random flip; returns 0 if the sampled term had no partner. */
static int flip(Term* t, int r) {
  const int i = rndn(r), p = rndn(3);
  int cand[RMAX], nc = 0;
  for (int j = 0; j < r; ++j)
    if (j != i && t[j].f[p] == t[i].f[p]) cand[nc++] = j;
  if (!nc) return 0;
  const int j = cand[rndn(nc)];
  int q = (p + 1) % 3, s = (p + 2) % 3;
  if (rnd() & 1) {
    const int x = q;
    q = s;
    s = x;
  }
  t[i].f[q] ^= t[j].f[q];
  t[j].f[s] ^= t[i].f[s];
  return 1;
}

/* Plus move on two terms (a, b, c), (a', b', c'):
 *   (a + a', b, c), (a', b + b', c), (a', b', c + c')
 * (one term more; the sum is unchanged, and no two of the three share two
 * factors, so the next reduction does not undo it).  The roles of the three
 * factors are rotated at random. */
static void plus(Term* t, int* r) {
  if (*r + 1 >= RMAX || *r < 2) return;
  const int i = rndn(*r);
  int j = rndn(*r - 1);
  if (j >= i) ++j;
  const int p = rndn(3), q = (p + 1) % 3, s = (p + 2) % 3;
  const Term x = t[i], y = t[j];
  Term u = x, v = y, w = y;
  u.f[p] = x.f[p] ^ y.f[p];          /* (a + a', b, c)   */
  v.f[q] = x.f[q] ^ y.f[q];          /* (a', b + b', c)  */
  v.f[s] = x.f[s];
  w.f[s] = x.f[s] ^ y.f[s];          /* (a', b', c + c') */
  t[i] = u;
  t[j] = v;
  t[(*r)++] = w;
}

static void print_scheme(const Term* t, int r) {
  printf("%d\n", r);
  for (int p = 0; p < r; ++p) printf("%u %u %u\n", t[p].f[0], t[p].f[1], t[p].f[2]);
}

int main(void) {
  int target;
  long long max_steps, plateau;
  unsigned long long seed;
  if (scanf("%d %d %d %d %lld %lld %llu", &n1, &n2, &n3, &target, &max_steps, &plateau, &seed) != 7) return 2;
  if (n1 < 1 || n1 > 16 || n2 < 1 || n2 > 16 || n3 < 1 || n3 > 32) return 2;
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n2; ++j)
      if (scanf("%u", &T[i][j]) != 1) return 2;
  Term best[RMAX], cur[RMAX];
  int rb;
  if (scanf("%d", &rb) != 1 || rb < 1 || rb > RMAX) return 2;
  for (int p = 0; p < rb; ++p)
    if (scanf("%u %u %u", &best[p].f[0], &best[p].f[1], &best[p].f[2]) != 3) return 2;
  if (!check(best, rb)) {
    fprintf(stderr, "starting scheme is wrong\n");
    return 3;
  }
  rng_state = seed * 0x9E3779B97F4A7C15ull + 1;
  reduce_all(best, &rb);
  memcpy(cur, best, sizeof(Term) * rb);
  int r = rb;
  long long since = 0;
  for (long long step = 0; step < max_steps && rb > target; ++step) {
    if (!flip(cur, r)) continue;
    reduce_all(cur, &r);
    ++since;
    if (r < rb) {
      if (!check(cur, r)) {
        fprintf(stderr, "internal error: flip broke the scheme\n");
        return 4;
      }
      rb = r;
      memcpy(best, cur, sizeof(Term) * r);
      since = 0;
      fprintf(stderr, "step %lld: rank %d\n", step, rb);
    } else if (since > plateau) {
      /* restart from the best scheme, with one plus move half of the time */
      memcpy(cur, best, sizeof(Term) * rb);
      r = rb;
      if (rnd() & 1) plus(cur, &r);
      since = 0;
    } else if (r > rb + 2) {
      memcpy(cur, best, sizeof(Term) * rb);
      r = rb;
    }
  }
  if (!check(best, rb)) return 4;
  print_scheme(best, rb);
  return 0;
}
