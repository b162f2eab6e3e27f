// Bit-slice helpers of the panel kernels (echelon.cu, ple.cu): a row's
// entries over 32 columns held as E 32-bit words, word t holding coefficient
// t of every entry (Section 3.2), and field arithmetic on them.
#pragma once
#include <cstdint>

namespace m4rie {
namespace bitslice {

// a * x modulo f (flow: f without its x^E term)
template <int E>
__device__ __forceinline__ uint32_t times_x(uint32_t a, uint32_t flow) {
  return (a << 1) ^ (((a >> (E - 1)) & 1u) ? (flow | (1u << E)) : 0u);
}

// sl += s * p on bit slices (s a field element; slice t of p at
// p[t * stride]): slice t of p carries x^t, so it adds with the slices of
// s x^t.
template <int E>
__device__ __forceinline__ void add_scaled(uint32_t (&sl)[E], uint32_t s, const uint32_t* p, int stride,
                                           uint32_t flow) {
#pragma unroll
  for (int t = 0; t < E; ++t) {
    const uint32_t pt = p[t * stride];
#pragma unroll
    for (int s2 = 0; s2 < E; ++s2) sl[s2] ^= pt & (0u - ((s >> s2) & 1u));
    s = times_x<E>(s, flow);
  }
}

// out = s * in on bit slices held in registers.
template <int E>
__device__ __forceinline__ void scaled(uint32_t (&out)[E], uint32_t s, const uint32_t (&in)[E], uint32_t flow) {
#pragma unroll
  for (int t = 0; t < E; ++t) out[t] = 0;
#pragma unroll
  for (int t = 0; t < E; ++t) {
#pragma unroll
    for (int s2 = 0; s2 < E; ++s2) out[s2] ^= in[t] & (0u - ((s >> s2) & 1u));
    s = times_x<E>(s, flow);
  }
}

// The element at bit b of the slices.
template <int E>
__device__ __forceinline__ uint32_t element_at(const uint32_t (&sl)[E], int b) {
  uint32_t v = 0;
#pragma unroll
  for (int t = 0; t < E; ++t) v |= ((sl[t] >> b) & 1u) << t;
  return v;
}

// The 32 elements src[0 .. 32) (panel columns cbase .. cbase+31; those
// outside [lo, hi) read as 0) as E bit slices; all loads are issued before
// any is used.  Returns whether an entry was >= 2^E.
template <typename T, int E>
__device__ __forceinline__ bool load_word(const T* __restrict__ src, int cbase, int lo, int hi, uint32_t (&sl)[E]) {
  const uint32_t q = (1u << E) - 1;
  uint32_t v[32];
#pragma unroll
  for (int b = 0; b < 32; ++b) {
    const int c = cbase + b;
    v[b] = (c >= lo && c < hi) ? (uint32_t)src[b] : 0u;
  }
  uint32_t any = 0;
#pragma unroll
  for (int t = 0; t < E; ++t) sl[t] = 0;
#pragma unroll
  for (int b = 0; b < 32; ++b) {
    any |= v[b];
#pragma unroll
    for (int t = 0; t < E; ++t) sl[t] |= ((v[b] >> t) & 1u) << b;
  }
  return (any & ~q) != 0;
}

}  // namespace bitslice
}  // namespace m4rie
