// PT2 importance of candidate determinants (Step 2, Eq. pt2_score):
//   v(x)   = <x|H|Psi0> = sum_{J in subspace} <x|H|J> c_J,
//   H_xx   = <x|H|x>,
//   s(x)   = v(x)^2 / |E0 - H_xx|,
// for candidates x = (x_alpha, x_beta) inside or outside the product subspace (an
// "external sigma").  <x|H|J> is non-zero only when J differs from x by at most two
// spin-orbital excitations, so with J = (J_a, J_b) the terms are
//   (0,0) J = x                                  H_xx c_x           (x in the subspace)
//   (1,0),(2,0) J_b = x_b, J_a linked to x_a      alpha single/double element
//   (0,1),(0,2) J_a = x_a, J_b linked to x_b      beta single/double element
//   (1,1) J_a, J_b singles of x_a, x_b            sign_a sign_b (pq|rs)
// One warp per candidate: it scans S_alpha and S_beta with XOR/popcount, adds the
// terms whose partner string is x's own (found by binary search) on the fly, keeps
// the single links of both sides in shared memory (at most n_e (n - n_e) each) and
// then sums the single x single products.  FP64 throughout.
//
// Element conventions (bra = the candidate's string J, ket = the subspace string I,
// J = sign a+_p a_q I for a single, J = sign a+_p a+_r a_s a_q I for a double with
// holes q < s and particles p < r; sign by applying the operators to I in turn):
//   single:  sign [h_pq + sum_{j in I, j != q} ((pq|jj) - (pj|jq))
//                  + sum_{j in other-spin string} (pq|jj)]
//   double:  sign [(pq|rs) - (ps|rq)]
#include <algorithm>

#include "hinqs_internal.cuh"
#include "slater.cuh"

namespace hinqs {

namespace {

using namespace slater;
constexpr int kPt2Warps = 4;

__device__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct Pt2Args {
  int n, na, nb;
  double e_nuc, e0;
  const double* h;
  const double* eri;
  const uint64_t* sa;
  const uint64_t* sb;
  int64_t Na, Nb;
  const double* c;
  const uint64_t* xa;
  const uint64_t* xb;
  int64_t M;
  double* v;
  double* hxx;
  double* score;
  unsigned int* bad;  // candidates with a wrong electron count
  int cap_a, cap_b;   // single-link capacities n_a (n - n_a), n_b (n - n_b)
};

// scan one spin's strings for links of x (same electron count); adds the terms with
// the other spin fixed at x's own string (index fixed_other >= 0) and records singles
__device__ void scan_side(const Pt2Args& A, const uint64_t* __restrict__ S, int64_t NS,
                          uint64_t x, uint64_t x_other, int64_t fixed_other, bool alpha,
                          int2* list, int* count, double& acc) {
  const int lane = threadIdx.x & 31;
  for (int64_t i0 = 0; i0 < NS; i0 += 32) {
    const int64_t i = i0 + lane;
    int d = 8;
    uint64_t I = 0;
    if (i < NS) {
      I = S[i];
      d = __popcll(I ^ x);
    }
    const unsigned m = __ballot_sync(0xffffffffu, d == 2);
    int p = 0, q = 0;
    if (d == 2) {
      q = __ffsll((long long)(I & ~x)) - 1;  // hole in the ket I
      p = __ffsll((long long)(x & ~I)) - 1;  // particle in the bra x
      const int slot = *count + __popc(m & ((1u << lane) - 1u));
      const int sg = single_sign(I, p, q);
      list[slot] = make_int2((int)i, sg * (p * A.n + q + 1));
    }
    if (fixed_other >= 0 && (d == 2 || d == 4)) {
      const double e = (d == 2) ? single_elem(A.h, A.eri, A.n, I, x_other, p, q)
                                : double_elem(A.eri, A.n, I, x);
      const int64_t J = alpha ? i * A.Nb + fixed_other : fixed_other * A.Nb + i;
      acc += e * A.c[J];
    }
    __syncwarp();
    if (lane == 0) *count += __popc(m);
    __syncwarp();
  }
}

__global__ void __launch_bounds__(32 * kPt2Warps) k_pt2(Pt2Args A) {
  extern __shared__ int2 lists[];  // per warp: cap_a alpha singles, cap_b beta singles
  __shared__ int counts[kPt2Warps][2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int2* la = lists + (size_t)warp * (A.cap_a + A.cap_b);
  int2* lb = la + A.cap_a;
  const int n = A.n;
  const uint64_t valid = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
  for (int64_t k = (int64_t)blockIdx.x * kPt2Warps + warp; k < A.M;
       k += (int64_t)gridDim.x * kPt2Warps) {
    const uint64_t xa = A.xa[k], xb = A.xb[k];
    if (__popcll(xa) != A.na || __popcll(xb) != A.nb || (xa & ~valid) || (xb & ~valid)) {
      if (lane == 0) {
        atomicAdd(A.bad, 1u);
        A.v[k] = A.hxx[k] = A.score[k] = __longlong_as_double(0x7ff8000000000000ll);
      }
      continue;
    }
    // H_xx: one- and two-body diagonal over the occupied orbitals of both strings
    double hd = 0.0;
    for (int ij = lane; ij < n * n; ij += 32) {
      const int i = ij / n, j = ij % n;
      const bool ia = (xa >> i) & 1, ib = (xb >> i) & 1, ja = (xa >> j) & 1, jb = (xb >> j) & 1;
      if (i == j) hd += (ia + ib) * A.h[i * n + i];
      const double J = eri4(A.eri, n, i, i, j, j), K = eri4(A.eri, n, i, j, j, i);
      if (ia && ja) hd += 0.5 * (J - K);
      if (ib && jb) hd += 0.5 * (J - K);
      if (ia && jb) hd += J;
    }
    hd = warp_sum(hd) + A.e_nuc;
    const int64_t ia0 = find_string(A.sa, A.Na, xa), ib0 = find_string(A.sb, A.Nb, xb);
    double acc = 0.0;
    if (lane == 0 && ia0 >= 0 && ib0 >= 0) acc += hd * A.c[ia0 * A.Nb + ib0];
    if (lane == 0) counts[warp][0] = counts[warp][1] = 0;
    __syncwarp();
    scan_side(A, A.sa, A.Na, xa, xb, ib0, true, la, &counts[warp][0], acc);
    scan_side(A, A.sb, A.Nb, xb, xa, ia0, false, lb, &counts[warp][1], acc);
    // single x single: sign_a sign_b (pq|rs) c(J_a, J_b)
    const int na1 = counts[warp][0], nb1 = counts[warp][1];
    const int64_t npair = (int64_t)na1 * nb1;
    for (int64_t t = lane; t < npair; t += 32) {
      const int2 a = la[t / nb1], b = lb[t % nb1];
      const int pqa = (a.y > 0 ? a.y : -a.y) - 1, rsb = (b.y > 0 ? b.y : -b.y) - 1;
      const double e = A.eri[(int64_t)pqa * n * n + rsb];
      const double sg = ((a.y > 0) == (b.y > 0)) ? 1.0 : -1.0;
      acc += sg * e * A.c[(int64_t)a.x * A.Nb + b.x];
    }
    acc = warp_sum(acc);
    if (lane == 0) {
      A.v[k] = acc;
      A.hxx[k] = hd;
      A.score[k] = acc * acc / fabs(A.e0 - hd);
    }
    __syncwarp();
  }
}

}  // namespace

}  // namespace hinqs

using namespace hinqs;

extern "C" int hinqs_pt2_score(const hinqs_ham* H, const hinqs_subspace* B, const double* c,
                               double e0, const uint64_t* xa, const uint64_t* xb, int64_t m,
                               double* v, double* hxx, double* score, void* stream) {
  if (!H || !B) return fail(HINQS_ERR_ARG, "hinqs_pt2_score: NULL handle");
  if (m < 0 || (m > 0 && (!c || !xa || !xb || !v || !hxx || !score)))
    return fail(HINQS_ERR_ARG, "hinqs_pt2_score: NULL array or negative count");
  if (H->n != B->n || H->n_alpha != B->n_alpha || H->n_beta != B->n_beta)
    return fail(HINQS_ERR_ARG, "hinqs_pt2_score: Hamiltonian and subspace disagree");
  if (m == 0) return HINQS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  Pt2Args A;
  A.n = H->n;
  A.na = H->n_alpha;
  A.nb = H->n_beta;
  A.e_nuc = H->e_nuc;
  A.e0 = e0;
  A.h = H->h;
  A.eri = H->eri;
  A.sa = B->sa;
  A.sb = B->sb;
  A.Na = B->Na;
  A.Nb = B->Nb;
  A.c = c;
  A.xa = xa;
  A.xb = xb;
  A.M = m;
  A.v = v;
  A.hxx = hxx;
  A.score = score;
  A.cap_a = std::max(1, A.na * (A.n - A.na));
  A.cap_b = std::max(1, A.nb * (A.n - A.nb));
  const size_t smem = (size_t)kPt2Warps * (A.cap_a + A.cap_b) * sizeof(int2);
  unsigned int* bad = nullptr;
  HQ_TRY(dalloc(&bad, 1, s));
  A.bad = bad;
  int rc = HINQS_OK;
  auto run = [&]() -> int {
    HQ_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned int), s));
    if (smem > 48 * 1024) HQ_TRY(allow_max_smem(k_pt2));
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(m, kPt2Warps), 32 * kNumSMs);
    k_pt2<<<grid, 32 * kPt2Warps, smem, s>>>(A);
    HQ_LAUNCH_CHECK();
    unsigned int hb = 0;
    HQ_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, s));
    HQ_CUDA(cudaStreamSynchronize(s));
    if (hb)
      return fail(HINQS_ERR_PARTICLE_NUMBER,
                  "hinqs_pt2_score: %u candidates with a wrong electron count (outputs NaN)", hb);
    return HINQS_OK;
  };
  rc = run();
  dfree(bad, s);
  return rc;
}
