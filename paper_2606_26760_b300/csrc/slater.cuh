// Slater-Condon elements between two strings of one spin (device helpers shared by
// the kernels that meet determinants outside the subspace: PT2 scores, expansion).
// Conventions: bra J, ket I; a single is J = sign a+_p a_q I (p particle, q hole),
// a double J = sign a+_p a+_r a_s a_q I with holes q < s and particles p < r; the
// sign comes from applying the operators to I in turn.
//   single:  sign [h_pq + sum_{j in I, j != q} ((pq|jj) - (pj|jq))
//                  + sum_{j in other-spin string} (pq|jj)]
//   double:  sign [(pq|rs) - (ps|rq)]
//   alpha single x beta single: sign_a sign_b (p_a q_a | p_b q_b)
#pragma once
#include <cstdint>

namespace hinqs {
namespace slater {

__device__ __forceinline__ int parity_below(uint64_t t, int k) {
  return __popcll(t & ((1ull << k) - 1ull)) & 1;
}

// sign of a+_p a_q applied to I (q in I, p not in I \ {q})
__device__ __forceinline__ int single_sign(uint64_t I, int p, int q) {
  int par = parity_below(I, q);
  const uint64_t t = I & ~(1ull << q);
  par ^= parity_below(t, p);
  return par ? -1 : 1;
}

// sign of a+_p a+_r a_s a_q applied to I (applied right to left)
__device__ __forceinline__ int double_sign(uint64_t I, int p, int q, int r, int s) {
  uint64_t t = I;
  int par = parity_below(t, q);
  t &= ~(1ull << q);
  par ^= parity_below(t, s);
  t &= ~(1ull << s);
  par ^= parity_below(t, r);
  t |= 1ull << r;
  par ^= parity_below(t, p);
  return par ? -1 : 1;
}

__device__ __forceinline__ double eri4(const double* __restrict__ eri, int n, int p, int q, int r,
                                       int s) {
  return eri[((int64_t)(p * n + q) * n + r) * n + s];
}

// <J|H|I> for one spin with J = single excitation of I (p = particle, q = hole);
// `other` is the other spin's (unchanged) string
__device__ inline double single_elem(const double* __restrict__ h, const double* __restrict__ eri, int n,
                              uint64_t I, uint64_t other, int p, int q) {
  double v = h[p * n + q];
  uint64_t o = I & ~(1ull << q);
  while (o) {
    const int j = __ffsll((long long)o) - 1;
    o &= o - 1;
    v += eri4(eri, n, p, q, j, j) - eri4(eri, n, p, j, j, q);
  }
  o = other;
  while (o) {
    const int j = __ffsll((long long)o) - 1;
    o &= o - 1;
    v += eri4(eri, n, p, q, j, j);
  }
  return single_sign(I, p, q) * v;
}

// <J|H|I> for one spin with J a double excitation of I
__device__ inline double double_elem(const double* __restrict__ eri, int n, uint64_t I, uint64_t J) {
  const uint64_t holes = I & ~J, parts = J & ~I;
  const int q = __ffsll((long long)holes) - 1, s = 63 - __clzll((long long)holes);
  const int p = __ffsll((long long)parts) - 1, r = 63 - __clzll((long long)parts);
  const double v = eri4(eri, n, p, q, r, s) - eri4(eri, n, p, s, r, q);
  return double_sign(I, p, q, r, s) * v;
}

// index of x in the ascending array S, or -1
__device__ inline int64_t find_string(const uint64_t* __restrict__ S, int64_t N, uint64_t x) {
  int64_t lo = 0, hi = N;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (S[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return (lo < N && S[lo] == x) ? lo : -1;
}

}  // namespace slater
}  // namespace hinqs
