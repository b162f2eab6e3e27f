// Host-side field helpers and GF(2)-product schedules (schedule.cpp).
#pragma once
#include <cstdint>
#include <vector>

namespace m4rie {

int poly_degree(uint32_t f);
bool poly_irreducible(uint32_t f);
uint32_t x_pow_mod(int e, uint32_t f, int d);

// alpha^j-B schedule: A masks 1 << j (j < e); B masks for plane (j, i) at
// bmask[i * e + j]: bit l set iff coefficient i of x^(j + l) mod f is 1.
void alpha_b_masks(int e, uint32_t f, uint16_t* amask, uint16_t* bmask);

struct Schedule {
  int e = 0, r = 0;
  std::vector<uint16_t> amask, bmask;  // per product: XOR-sum of slices on each side
  uint64_t out_mask[10];               // bit p of out_mask[s]: product p feeds output slice s
};

// Karatsuba-like schedule for degree e under f; false if it fails its check.
bool karatsuba_schedule(int e, uint32_t f, Schedule* out);

}  // namespace m4rie
