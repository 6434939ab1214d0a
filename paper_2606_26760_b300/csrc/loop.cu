// The outer loop of Sec. 2.2 around the subspace solve, on the device:
//   hinqs_select_top           Step 2 ranking: top K by s(x), or the K_0 lowest H_xx
//   hinqs_determinant_diag     H_xx of arbitrary determinants (Step 2 cold start)
//   hinqs_lookup_determinants  position of determinants in the product subspace
//   hinqs_candidate_pool       Steps 1 / 1': distinct candidates of the pooled
//                              proposals, particle-number filter, minus the basis
//   hinqs_basis_update         Step 2: cold start, full rescore, append with eviction
//   hinqs_remap_vector         Step 3 warm start: the previous eigenvector carried to
//                              the new product subspace
//   hinqs_nqs_loss             Step 4: teacher weights, advantages, the three loss
//                              terms and their gradient on a minibatch
// Selections are exact (radix selection on order-preserving keys, ties to the lower
// position), sets are sorted keys alpha << 32 | beta (n_orb < 32; above, the strings'
// ranks among the sorted distinct strings in play), and every sum is a fixed-shape
// tree, so results do not depend on scheduling.
#include <algorithm>

#include "hinqs_internal.cuh"
#include "slater.cuh"

namespace hinqs {

int check_triplet(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                  const hinqs_links_s* lb, const char* who);

namespace {

using namespace slater;
constexpr uint64_t kNoKey = ~0ull;
constexpr int kRedThreads = 256;

__device__ __forceinline__ bool string_ok(uint64_t x, int n, int ne) {
  return __popcll(x) == ne && (n >= 64 || (x >> n) == 0ull);
}

// <x|H|x> of the determinant (a, b): one-body terms, same-spin pairs i < j with
// (ii|jj) - (ij|ji), opposite-spin pairs with (ii|jj), plus E_nuc
__device__ double det_diag(const double* __restrict__ h, const double* __restrict__ eri, int n,
                           uint64_t a, uint64_t b, double e_nuc) {
  double v = e_nuc;
  for (int spin = 0; spin < 2; ++spin) {
    uint64_t o = spin ? b : a;
    while (o) {
      const int i = __ffsll((long long)o) - 1;
      o &= o - 1;
      v += h[i * n + i];
      uint64_t r = o;  // the occupied orbitals above i
      while (r) {
        const int j = __ffsll((long long)r) - 1;
        r &= r - 1;
        v += eri4(eri, n, i, i, j, j) - eri4(eri, n, i, j, j, i);
      }
    }
  }
  uint64_t oa = a;
  while (oa) {
    const int i = __ffsll((long long)oa) - 1;
    oa &= oa - 1;
    uint64_t ob = b;
    while (ob) {
      const int j = __ffsll((long long)ob) - 1;
      ob &= ob - 1;
      v += eri4(eri, n, i, i, j, j);
    }
  }
  return v;
}

__global__ void k_det_diag(const double* __restrict__ h, const double* __restrict__ eri, int n,
                           int na, int nb, double e_nuc, const uint64_t* __restrict__ xa,
                           const uint64_t* __restrict__ xb, int64_t m, double* __restrict__ hxx,
                           unsigned int* bad) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = xa[k], b = xb[k];
    if (string_ok(a, n, na) && string_ok(b, n, nb)) {
      hxx[k] = det_diag(h, eri, n, a, b, e_nuc);
    } else {
      hxx[k] = __longlong_as_double(0x7ff8000000000000ll);
      atomicAdd(bad, 1u);
    }
  }
}

__global__ void k_lookup(const uint64_t* __restrict__ sa, int64_t Na, const uint64_t* __restrict__ sb,
                         int64_t Nb, const uint64_t* __restrict__ xa, const uint64_t* __restrict__ xb,
                         int64_t m, int64_t* __restrict__ idx) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ia = find_string(sa, Na, xa[k]);
    const int64_t ib = ia >= 0 ? find_string(sb, Nb, xb[k]) : -1;
    idx[k] = (ia >= 0 && ib >= 0) ? ia * Nb + ib : -1;
  }
}

// ---------------------------------------------------------------- candidate pool

// keys of the pooled proposals (first list, then second), kNoKey for padding and for
// entries that fail the particle-number filter (counted in *dropped)
__global__ void k_pool_keys(const uint64_t* __restrict__ xa1, const uint64_t* __restrict__ xb1,
                            int64_t m1, const uint64_t* __restrict__ xa2,
                            const uint64_t* __restrict__ xb2, int64_t m2, int n, int na, int nb,
                            uint64_t* __restrict__ keys, int64_t m_pad,
                            unsigned long long* dropped) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t a, b;
    if (i < m1) {
      a = xa1[i];
      b = xb1[i];
    } else if (i < m1 + m2) {
      a = xa2[i - m1];
      b = xb2[i - m1];
    } else {
      keys[i] = kNoKey;
      continue;
    }
    const bool ok = string_ok(a, n, na) && string_ok(b, n, nb);
    keys[i] = ok ? ((a << 32) | b) : kNoKey;
    if (!ok) atomicAdd(dropped, 1ull);
  }
}

// n_orb >= 32: the key of a determinant is (rank of alpha) << 32 | (rank of beta) in
// the sorted distinct strings of the proposals (ranks keep the strings' order), so that
// any n_orb <= 64 packs into 64 bits; a string outside its dictionary gives kNoKey
__device__ __forceinline__ uint64_t rank_key(const uint64_t* __restrict__ DA, int64_t ua,
                                             const uint64_t* __restrict__ DB, int64_t ub,
                                             uint64_t a, uint64_t b) {
  const int64_t ra = find_string(DA, ua, a), rb = ra >= 0 ? find_string(DB, ub, b) : -1;
  return (ra >= 0 && rb >= 0) ? (((uint64_t)ra << 32) | (uint64_t)rb) : kNoKey;
}

__global__ void k_pool_rank_keys(const uint64_t* __restrict__ xa1,
                                 const uint64_t* __restrict__ xb1, int64_t m1,
                                 const uint64_t* __restrict__ xa2,
                                 const uint64_t* __restrict__ xb2, int64_t m2, int n, int na,
                                 int nb, const uint64_t* __restrict__ DA, int64_t ua,
                                 const uint64_t* __restrict__ DB, int64_t ub,
                                 uint64_t* __restrict__ keys, int64_t m_pad,
                                 unsigned long long* dropped) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t a, b;
    if (i < m1) {
      a = xa1[i];
      b = xb1[i];
    } else if (i < m1 + m2) {
      a = xa2[i - m1];
      b = xb2[i - m1];
    } else {
      keys[i] = kNoKey;
      continue;
    }
    const bool ok = string_ok(a, n, na) && string_ok(b, n, nb);
    keys[i] = ok ? rank_key(DA, ua, DB, ub, a, b) : kNoKey;
    if (!ok) atomicAdd(dropped, 1ull);
  }
}

__global__ void k_exclude_rank_keys(const uint64_t* __restrict__ ea,
                                    const uint64_t* __restrict__ eb, int64_t me,
                                    const uint64_t* __restrict__ DA, int64_t ua,
                                    const uint64_t* __restrict__ DB, int64_t ub,
                                    uint64_t* __restrict__ keys, int64_t m_pad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_pad;
       i += (int64_t)gridDim.x * blockDim.x)
    keys[i] = i < me ? rank_key(DA, ua, DB, ub, ea[i], eb[i]) : kNoKey;
}

__global__ void k_pool_rank_scatter(const uint64_t* __restrict__ keys, int64_t m_pad,
                                    const int64_t* __restrict__ flag,
                                    const int64_t* __restrict__ pos,
                                    const uint64_t* __restrict__ DA,
                                    const uint64_t* __restrict__ DB, uint64_t* __restrict__ ya,
                                    uint64_t* __restrict__ yb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_pad;
       i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) {
      ya[pos[i]] = DA[keys[i] >> 32];
      yb[pos[i]] = DB[keys[i] & 0xffffffffull];
    }
}

// keys of the excluded determinants; entries that cannot be a valid key (bits at or
// above 32) become kNoKey, which matches no candidate
__global__ void k_exclude_keys(const uint64_t* __restrict__ ea, const uint64_t* __restrict__ eb,
                               int64_t me, uint64_t* __restrict__ keys, int64_t m_pad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = kNoKey;
    if (i < me && (ea[i] >> 32) == 0ull && (eb[i] >> 32) == 0ull) k = (ea[i] << 32) | eb[i];
    keys[i] = k;
  }
}

__device__ __forceinline__ bool key_in(const uint64_t* __restrict__ S, int64_t N, uint64_t x) {
  int64_t lo = 0, hi = N;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (S[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo < N && S[lo] == x;
}

// flag the first copy of every valid key that is not excluded (keys sorted)
__global__ void k_pool_flags(const uint64_t* __restrict__ keys, int64_t m_pad,
                             const uint64_t* __restrict__ ex, int64_t ex_pad,
                             int64_t* __restrict__ flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    flag[i] = (k != kNoKey && (i == 0 || k != keys[i - 1]) && !(ex && key_in(ex, ex_pad, k)))
                  ? 1 : 0;
  }
}

__global__ void k_pool_scatter(const uint64_t* __restrict__ keys, int64_t m_pad,
                               const int64_t* __restrict__ flag, const int64_t* __restrict__ pos,
                               uint64_t* __restrict__ ya, uint64_t* __restrict__ yb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_pad;
       i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) {
      ya[pos[i]] = keys[i] >> 32;
      yb[pos[i]] = keys[i] & 0xffffffffull;
    }
}

// ------------------------------------------------------------------ basis update

// out[j] = pool entry sel[j] (sel NULL: entry j), j < cnt; pool entry p is segment-1
// entry p when p < n1, else segment-2 entry map2[p - n1] (map2 NULL: p - n1).
// oa / ob may be NULL (scores only).
__global__ void k_gather_pool(const int64_t* __restrict__ sel, int64_t cnt,
                              const uint64_t* __restrict__ a1, const uint64_t* __restrict__ b1,
                              const double* __restrict__ s1, int64_t n1,
                              const uint64_t* __restrict__ a2, const uint64_t* __restrict__ b2,
                              const double* __restrict__ s2, const int64_t* __restrict__ map2,
                              uint64_t* __restrict__ oa, uint64_t* __restrict__ ob,
                              double* __restrict__ os) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cnt;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = sel ? sel[j] : j;
    if (p < n1) {
      if (oa) oa[j] = a1[p];
      if (ob) ob[j] = b1[p];
      os[j] = s1[p];
    } else {
      const int64_t q = map2 ? map2[p - n1] : p - n1;
      if (oa) oa[j] = a2[q];
      if (ob) ob[j] = b2[q];
      os[j] = s2[q];
    }
  }
}

// ------------------------------------------------------------------ warm start

__global__ void k_map_strings(const uint64_t* __restrict__ s_new, int64_t n_new,
                              const uint64_t* __restrict__ s_old, int64_t n_old,
                              int64_t* __restrict__ map) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_new;
       i += (int64_t)gridDim.x * blockDim.x)
    map[i] = find_string(s_old, n_old, s_new[i]);
}

__global__ void k_remap(const double* __restrict__ c_old, int64_t Nb_old,
                        const int64_t* __restrict__ ma, const int64_t* __restrict__ mb, int64_t Na,
                        int64_t Nb, double* __restrict__ c_new) {
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < Na * Nb;
       I += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ia = I / Nb, ib = I - ia * Nb;
    const int64_t oa = ma[ia], ob = mb[ib];
    c_new[I] = (oa >= 0 && ob >= 0) ? c_old[oa * Nb_old + ob] : 0.0;
  }
}

// ------------------------------------------------------------------ reductions

// tree sum of one value per thread over a block of kRedThreads threads (fixed shape)
__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = kRedThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void k_sumsq_partials(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += x[i] * x[i];
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// out[c] = sum_b part[b * width + c] for c < width, one block
__global__ void k_sum_partials(const double* __restrict__ part, int nblk, int width,
                               double* __restrict__ out) {
  __shared__ double sh[kRedThreads];
  for (int c = 0; c < width; ++c) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += part[(int64_t)b * width + c];
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) out[c] = t;
  }
}

// ---------------------------------------------------------------- NQS loss inputs

// z[0] = sum over the basis of p_alpha(x_a) p_beta(x_b): the whole product
// (basis NULL: (sum p_alpha)(sum p_beta)) or the listed product indices
__global__ void k_teacher_norm_partials(const double* __restrict__ pa, int64_t Na,
                                        const double* __restrict__ pb, int64_t Nb,
                                        const int64_t* __restrict__ basis, int64_t n_basis,
                                        double* __restrict__ part, unsigned int* bad) {
  __shared__ double sh[kRedThreads];
  double x = 0.0, y = 0.0;
  if (basis) {
    const int64_t N = Na * Nb;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_basis;
         k += (int64_t)gridDim.x * blockDim.x) {
      const int64_t I = basis[k];
      if (I < 0 || I >= N) {
        atomicAdd(bad, 1u);
        continue;
      }
      x += pa[I / Nb] * pb[I % Nb];
    }
    const double t = block_sum(x, sh);
    if (threadIdx.x == 0) {  // second factor 1: summed over the blocks it stays 1
      part[2 * blockIdx.x] = t;
      part[2 * blockIdx.x + 1] = blockIdx.x == 0 ? 1.0 : 0.0;
    }
  } else {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Na;
         i += (int64_t)gridDim.x * blockDim.x)
      x += pa[i];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Nb;
         i += (int64_t)gridDim.x * blockDim.x)
      y += pb[i];
    const double tx = block_sum(x, sh);
    const double ty = block_sum(y, sh);
    if (threadIdx.x == 0) {
      part[2 * blockIdx.x] = tx;
      part[2 * blockIdx.x + 1] = ty;
    }
  }
}

struct LossArgs {
  int n;
  double e_nuc, e0;
  const double* pa;
  const double* pb;
  const double* ha;   // same-spin diagonal per alpha string
  const double* hb;   // same-spin diagonal per beta string
  const double* Va;   // [N_a][n*n] sum_{i in I_a} (ii|xy)
  const uint64_t* sb;
  int64_t Na, Nb;
  const int64_t* batch;
  int64_t m;
  const double* log_pi;
  double ct, ce, cs;
  const double* zsum;  // [2]: the teacher normaliser is zsum[0] * zsum[1]
  double* w;
  double* adv;
  double* grad;
  double* part;        // [gridDim][3]
  unsigned int* bad;
};

__global__ void k_nqs_loss(LossArgs A) {
  __shared__ double sh[kRedThreads];
  const double Z = A.zsum[0] * A.zsum[1];
  const int64_t N = A.Na * A.Nb;
  const int n2 = A.n * A.n;
  const double inv_m = 1.0 / (double)A.m;
  double lt = 0.0, le = 0.0, ls = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < A.m;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = A.batch[j];
    if (I < 0 || I >= N) {
      const double nan = __longlong_as_double(0x7ff8000000000000ll);
      A.w[j] = nan;
      A.adv[j] = nan;
      A.grad[j] = nan;
      atomicAdd(A.bad, 1u);
      continue;
    }
    const int64_t ia = I / A.Nb, ib = I - ia * A.Nb;
    const double wx = A.pa[ia] * A.pb[ib] / Z;
    double hxx = A.ha[ia] + A.hb[ib] + A.e_nuc;
    uint64_t occ = A.sb[ib];
    while (occ) {
      const int q = __ffsll((long long)occ) - 1;
      occ &= occ - 1;
      hxx += A.Va[ia * n2 + q * A.n + q];
    }
    const double ax = hxx - A.e0;
    const double lp = A.log_pi[j];
    A.w[j] = wx;
    A.adv[j] = ax;
    A.grad[j] = -A.ct * wx + A.ce * wx * ax + A.cs * inv_m;
    lt -= wx * lp;
    le += wx * ax * lp;
    ls += lp;
  }
  const double t0 = block_sum(lt, sh);
  const double t1 = block_sum(le, sh);
  const double t2 = block_sum(ls, sh);
  if (threadIdx.x == 0) {
    A.part[3 * blockIdx.x] = t0;
    A.part[3 * blockIdx.x + 1] = t1;
    A.part[3 * blockIdx.x + 2] = t2;
  }
}

// loss = (total, teacher, energy, entropy) from the summed terms
__global__ void k_nqs_loss_final(const double* __restrict__ sums, int64_t m, double ct, double ce,
                                 double cs, double* __restrict__ loss) {
  const double lt = sums[0], le = sums[1], ls = sums[2] / (double)m;
  loss[0] = ct * lt + ce * le + cs * ls;
  loss[1] = lt;
  loss[2] = le;
  loss[3] = ls;
}

unsigned grid_for(int64_t n, int64_t cap = 16 * kNumSMs) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), cap));
}

int64_t pow2_at_least(int64_t m) {
  int64_t p = 2;
  while (p < m) p <<= 1;
  return p;
}

bool same_sector(const hinqs_subspace_s* x, const hinqs_subspace_s* y) {
  return x->n == y->n && x->n_alpha == y->n_alpha && x->n_beta == y->n_beta;
}

}  // namespace
}  // namespace hinqs

using namespace hinqs;

extern "C" int hinqs_select_top(const double* values, int64_t m, int64_t k, int largest,
                                int64_t* idx_out, void* stream) {
  if (m < 0 || k < 0 || (m > 0 && !values) || (k > 0 && m > 0 && !idx_out))
    return fail(HINQS_ERR_ARG, "hinqs_select_top: NULL argument or negative size");
  return select_top_impl(values, m, k, largest ? kSelLargest : kSelSmallest, idx_out,
                         (cudaStream_t)stream);
}

extern "C" int hinqs_determinant_diag(const hinqs_ham* H, const uint64_t* xa, const uint64_t* xb,
                                      int64_t m, double* hxx, void* stream) {
  if (!H || m < 0 || (m > 0 && (!xa || !xb || !hxx)))
    return fail(HINQS_ERR_ARG, "hinqs_determinant_diag: NULL argument or negative m");
  if (m == 0) return HINQS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned int* bad = nullptr;
  HQ_TRY(dalloc(&bad, 1, s));
  auto run = [&]() -> int {
    HQ_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned int), s));
    k_det_diag<<<grid_for(m), 256, 0, s>>>(H->h, H->eri, H->n, H->n_alpha, H->n_beta, H->e_nuc,
                                           xa, xb, m, hxx, bad);
    HQ_LAUNCH_CHECK();
    unsigned int hb = 0;
    HQ_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, s));
    HQ_CUDA(cudaStreamSynchronize(s));
    if (hb)
      return fail(HINQS_ERR_PARTICLE_NUMBER,
                  "hinqs_determinant_diag: %u determinants with a wrong electron count (outputs NaN)",
                  hb);
    return HINQS_OK;
  };
  const int rc = run();
  dfree(bad, s);
  return rc;
}

extern "C" int hinqs_lookup_determinants(const hinqs_subspace* B, const uint64_t* xa,
                                         const uint64_t* xb, int64_t m, int64_t* idx, void* stream) {
  if (!B || m < 0 || (m > 0 && (!xa || !xb || !idx)))
    return fail(HINQS_ERR_ARG, "hinqs_lookup_determinants: NULL argument or negative m");
  if (m == 0) return HINQS_OK;
  k_lookup<<<grid_for(m), 256, 0, (cudaStream_t)stream>>>(B->sa, B->Na, B->sb, B->Nb, xa, xb, m,
                                                          idx);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

extern "C" int hinqs_candidate_pool(const hinqs_ham* H, const uint64_t* xa1, const uint64_t* xb1,
                                    int64_t m1, const uint64_t* xa2, const uint64_t* xb2,
                                    int64_t m2, const uint64_t* ea, const uint64_t* eb, int64_t me,
                                    uint64_t* ya, uint64_t* yb, int64_t cap, int64_t* count,
                                    int64_t* n_dropped, void* stream) {
  if (!H || !count || m1 < 0 || m2 < 0 || me < 0 || (m1 > 0 && (!xa1 || !xb1)) ||
      (m2 > 0 && (!xa2 || !xb2)) || (me > 0 && (!ea || !eb)))
    return fail(HINQS_ERR_ARG, "hinqs_candidate_pool: NULL argument or negative size");
  if (H->n_alpha == 64 || H->n_beta == 64)
    return fail(HINQS_ERR_ARG, "hinqs_candidate_pool: 64 electrons of one spin are not supported");
  *count = 0;
  if (n_dropped) *n_dropped = 0;
  const int64_t m = m1 + m2;
  if (m == 0) return HINQS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t m_pad = pow2_at_least(m);
  const int64_t ex_pad = me > 0 ? pow2_at_least(me) : 0;
  // n_orb <= 31: keys alpha << 32 | beta; else ranks in the proposals' distinct strings
  const bool ranks = H->n >= 32;
  uint64_t *keys = nullptr, *ex = nullptr, *DA = nullptr, *DB = nullptr, *tmp = nullptr;
  int64_t ua = 0, ub = 0;
  int64_t *flag = nullptr, *pos = nullptr;
  unsigned long long* dropped = nullptr;
  auto run = [&]() -> int {
    HQ_TRY(dalloc(&keys, m_pad, s));
    HQ_TRY(dalloc(&flag, m_pad, s));
    HQ_TRY(dalloc(&pos, m_pad, s));
    HQ_TRY(dalloc(&dropped, 1, s));
    HQ_CUDA(cudaMemsetAsync(dropped, 0, sizeof(unsigned long long), s));
    if (ranks) {
      // the dictionaries: sorted distinct valid alpha (beta) strings of both lists
      HQ_TRY(dalloc(&tmp, m, s));
      for (int spin = 0; spin < 2; ++spin) {
        const uint64_t* p1 = spin ? xb1 : xa1;
        const uint64_t* p2 = spin ? xb2 : xa2;
        if (m1) HQ_CUDA(cudaMemcpyAsync(tmp, p1, m1 * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        if (m2)
          HQ_CUDA(cudaMemcpyAsync(tmp + m1, p2, m2 * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        int64_t cnt = 0, drop = 0;
        const int r = build_species(tmp, m, H->n, spin ? H->n_beta : H->n_alpha, 0,
                                    spin ? &DB : &DA, &cnt, &drop, s);
        if (r < 0 && r != HINQS_ERR_EMPTY) return r;
        (spin ? ub : ua) = r < 0 ? 0 : cnt;
      }
      k_pool_rank_keys<<<grid_for(m_pad), 256, 0, s>>>(xa1, xb1, m1, xa2, xb2, m2, H->n,
                                                       H->n_alpha, H->n_beta, DA, ua, DB, ub,
                                                       keys, m_pad, dropped);
    } else {
      k_pool_keys<<<grid_for(m_pad), 256, 0, s>>>(xa1, xb1, m1, xa2, xb2, m2, H->n, H->n_alpha,
                                                  H->n_beta, keys, m_pad, dropped);
    }
    HQ_LAUNCH_CHECK();
    HQ_TRY(bitonic_sort(keys, m_pad, s));
    if (me > 0) {
      HQ_TRY(dalloc(&ex, ex_pad, s));
      if (ranks)
        k_exclude_rank_keys<<<grid_for(ex_pad), 256, 0, s>>>(ea, eb, me, DA, ua, DB, ub, ex, ex_pad);
      else
        k_exclude_keys<<<grid_for(ex_pad), 256, 0, s>>>(ea, eb, me, ex, ex_pad);
      HQ_LAUNCH_CHECK();
      HQ_TRY(bitonic_sort(ex, ex_pad, s));
    }
    k_pool_flags<<<grid_for(m_pad), 256, 0, s>>>(keys, m_pad, ex, ex_pad, flag);
    HQ_LAUNCH_CHECK();
    int64_t uniq = 0;
    HQ_TRY(exclusive_scan_i64(flag, pos, m_pad, &uniq, s));  // synchronises
    unsigned long long hd = 0;
    HQ_CUDA(cudaMemcpyAsync(&hd, dropped, sizeof(hd), cudaMemcpyDeviceToHost, s));
    HQ_CUDA(cudaStreamSynchronize(s));
    *count = uniq;
    if (n_dropped) *n_dropped = (int64_t)hd;
    if (!ya || !yb) return HINQS_OK;  // count only
    if (cap < uniq)
      return fail(HINQS_ERR_ARG, "hinqs_candidate_pool: cap %lld below the %lld candidates",
                  (long long)cap, (long long)uniq);
    if (ranks)
      k_pool_rank_scatter<<<grid_for(m_pad), 256, 0, s>>>(keys, m_pad, flag, pos, DA, DB, ya, yb);
    else
      k_pool_scatter<<<grid_for(m_pad), 256, 0, s>>>(keys, m_pad, flag, pos, ya, yb);
    HQ_LAUNCH_CHECK();
    return HINQS_OK;
  };
  const int rc = run();
  dfree(keys, s);
  dfree(ex, s);
  dfree(tmp, s);
  dfree(DA, s);
  dfree(DB, s);
  dfree(flag, s);
  dfree(pos, s);
  dfree(dropped, s);
  return rc;
}

extern "C" int hinqs_basis_update(int mode, const uint64_t* ba, const uint64_t* bb,
                                  const double* bs, int64_t nb, const uint64_t* ca,
                                  const uint64_t* cb, const double* cs, int64_t nc, int64_t k,
                                  int64_t b_max, uint64_t* oa, uint64_t* ob, double* os,
                                  int64_t cap, int64_t* n_out, void* stream) {
  if (!n_out || nb < 0 || nc < 0 || k < 0 || b_max < 0 || (nb > 0 && (!ba || !bb || !bs)) ||
      (nc > 0 && (!ca || !cb || !cs)))
    return fail(HINQS_ERR_ARG, "hinqs_basis_update: NULL argument or negative size");
  if (mode != HINQS_BASIS_COLD_START && mode != HINQS_BASIS_RESCORE && mode != HINQS_BASIS_APPEND)
    return fail(HINQS_ERR_ARG, "hinqs_basis_update: unknown mode %d", mode);
  cudaStream_t s = (cudaStream_t)stream;
  *n_out = 0;
  int64_t* sel = nullptr;
  int64_t* sel2 = nullptr;
  double* scores = nullptr;
  auto need_out = [&](int64_t cnt) -> int {
    if (cnt > 0 && (!oa || !ob || !os))
      return fail(HINQS_ERR_ARG, "hinqs_basis_update: NULL output");
    if (cap < cnt)
      return fail(HINQS_ERR_ARG, "hinqs_basis_update: cap %lld below the %lld basis entries",
                  (long long)cap, (long long)cnt);
    return HINQS_OK;
  };
  auto run = [&]() -> int {
    if (mode == HINQS_BASIS_COLD_START) {
      const int64_t kk = std::min(k, nc);
      HQ_TRY(need_out(kk));
      if (kk == 0) return HINQS_OK;
      HQ_TRY(dalloc(&sel, kk, s));
      HQ_TRY(select_top_impl(cs, nc, kk, kSelSmallest, sel, s));
      k_gather_pool<<<grid_for(kk), 256, 0, s>>>(sel, kk, ca, cb, cs, nc, nullptr, nullptr,
                                                 nullptr, nullptr, oa, ob, os);
      HQ_LAUNCH_CHECK();
      *n_out = kk;
      return HINQS_OK;
    }
    if (mode == HINQS_BASIS_RESCORE) {
      const int64_t np = nb + nc, kk = std::min(k, np);
      HQ_TRY(need_out(kk));
      if (kk == 0) return HINQS_OK;
      HQ_TRY(dalloc(&scores, np, s));
      if (nb) HQ_CUDA(cudaMemcpyAsync(scores, bs, nb * sizeof(double), cudaMemcpyDeviceToDevice, s));
      if (nc)
        HQ_CUDA(cudaMemcpyAsync(scores + nb, cs, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
      HQ_TRY(dalloc(&sel, kk, s));
      HQ_TRY(select_top_impl(scores, np, kk, kSelLargest, sel, s));
      k_gather_pool<<<grid_for(kk), 256, 0, s>>>(sel, kk, ba, bb, bs, nb, ca, cb, cs, nullptr, oa,
                                                 ob, os);
      HQ_LAUNCH_CHECK();
      *n_out = kk;
      return HINQS_OK;
    }
    // append the best k candidates, then evict the lowest-scored above b_max
    const int64_t k1 = std::min(k, nc), total = nb + k1;
    if (k1 > 0) {
      HQ_TRY(dalloc(&sel, k1, s));
      HQ_TRY(select_top_impl(cs, nc, k1, kSelLargest, sel, s));
    }
    if (b_max > 0 && total > b_max) {
      HQ_TRY(need_out(b_max));
      HQ_TRY(dalloc(&scores, total, s));
      k_gather_pool<<<grid_for(total), 256, 0, s>>>(nullptr, total, nullptr, nullptr, bs, nb,
                                                    nullptr, nullptr, cs, sel, nullptr, nullptr,
                                                    scores);
      HQ_LAUNCH_CHECK();
      HQ_TRY(dalloc(&sel2, b_max, s));
      HQ_TRY(select_top_impl(scores, total, b_max, kSelLargest, sel2, s));
      k_gather_pool<<<grid_for(b_max), 256, 0, s>>>(sel2, b_max, ba, bb, bs, nb, ca, cb, cs, sel,
                                                    oa, ob, os);
      HQ_LAUNCH_CHECK();
      *n_out = b_max;
      return HINQS_OK;
    }
    HQ_TRY(need_out(total));
    if (total > 0) {
      k_gather_pool<<<grid_for(total), 256, 0, s>>>(nullptr, total, ba, bb, bs, nb, ca, cb, cs,
                                                    sel, oa, ob, os);
      HQ_LAUNCH_CHECK();
    }
    *n_out = total;
    return HINQS_OK;
  };
  const int rc = run();
  dfree(sel, s);
  dfree(sel2, s);
  dfree(scores, s);
  if (rc < 0) *n_out = 0;
  return rc;
}

extern "C" int hinqs_remap_vector(const hinqs_subspace* old_sub, const double* c_old,
                                  const hinqs_subspace* new_sub, double* c_new, double* kept_norm2,
                                  void* stream) {
  if (!old_sub || !new_sub || !c_old || !c_new)
    return fail(HINQS_ERR_ARG, "hinqs_remap_vector: NULL argument");
  if (!same_sector(old_sub, new_sub))
    return fail(HINQS_ERR_ARG, "hinqs_remap_vector: the subspaces belong to different sectors");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t Na = new_sub->Na, Nb = new_sub->Nb, N = Na * Nb;
  int64_t *ma = nullptr, *mb = nullptr;
  double *part = nullptr, *tot = nullptr;
  auto run = [&]() -> int {
    HQ_TRY(dalloc(&ma, Na, s));
    HQ_TRY(dalloc(&mb, Nb, s));
    k_map_strings<<<grid_for(Na), 256, 0, s>>>(new_sub->sa, Na, old_sub->sa, old_sub->Na, ma);
    k_map_strings<<<grid_for(Nb), 256, 0, s>>>(new_sub->sb, Nb, old_sub->sb, old_sub->Nb, mb);
    k_remap<<<grid_for(N), 256, 0, s>>>(c_old, old_sub->Nb, ma, mb, Na, Nb, c_new);
    HQ_LAUNCH_CHECK();
    if (kept_norm2) {
      const unsigned g = grid_for(N, 4 * kNumSMs);
      HQ_TRY(dalloc(&part, g, s));
      HQ_TRY(dalloc(&tot, 1, s));
      k_sumsq_partials<<<g, kRedThreads, 0, s>>>(c_new, N, part);
      k_sum_partials<<<1, kRedThreads, 0, s>>>(part, (int)g, 1, tot);
      HQ_LAUNCH_CHECK();
      HQ_CUDA(cudaMemcpyAsync(kept_norm2, tot, sizeof(double), cudaMemcpyDeviceToHost, s));
      HQ_CUDA(cudaStreamSynchronize(s));
    }
    return HINQS_OK;
  };
  const int rc = run();
  dfree(ma, s);
  dfree(mb, s);
  dfree(part, s);
  dfree(tot, s);
  return rc;
}

extern "C" int hinqs_nqs_loss(const hinqs_ham* H, const hinqs_subspace* B, const hinqs_links* la,
                              const hinqs_links* lb, const double* p_alpha, const double* p_beta,
                              double e0, const int64_t* basis, int64_t n_basis,
                              const int64_t* batch, int64_t m, const double* log_pi,
                              const double* coef, double* w, double* adv, double* grad,
                              double* loss, void* stream) {
  HQ_TRY(check_triplet(H, B, la, lb, "hinqs_nqs_loss"));
  if (!p_alpha || !p_beta || !loss || m < 0 || n_basis < 0 || (basis && n_basis == 0) ||
      (m > 0 && (!batch || !log_pi || !w || !adv || !grad)))
    return fail(HINQS_ERR_ARG, "hinqs_nqs_loss: NULL argument or invalid size");
  if (m == 0) return fail(HINQS_ERR_ARG, "hinqs_nqs_loss: empty minibatch");
  cudaStream_t s = (cudaStream_t)stream;
  const double ct = coef ? coef[0] : 1.0, ce = coef ? coef[1] : 1.0, cs = coef ? coef[2] : 1.0;
  const unsigned gz = basis ? grid_for(n_basis, 4 * kNumSMs)
                            : grid_for(std::max(B->Na, B->Nb), 4 * kNumSMs);
  const unsigned gl = grid_for(m, 4 * kNumSMs);
  double *zpart = nullptr, *zsum = nullptr, *lpart = nullptr, *lsum = nullptr;
  unsigned int* bad = nullptr;
  auto run = [&]() -> int {
    HQ_TRY(dalloc(&zpart, 2 * (int64_t)gz, s));
    HQ_TRY(dalloc(&zsum, 2, s));
    HQ_TRY(dalloc(&lpart, 3 * (int64_t)gl, s));
    HQ_TRY(dalloc(&lsum, 3, s));
    HQ_TRY(dalloc(&bad, 1, s));
    HQ_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned int), s));
    k_teacher_norm_partials<<<gz, kRedThreads, 0, s>>>(p_alpha, B->Na, p_beta, B->Nb, basis,
                                                       n_basis, zpart, bad);
    k_sum_partials<<<1, kRedThreads, 0, s>>>(zpart, (int)gz, 2, zsum);
    LossArgs A;
    A.n = H->n;
    A.e_nuc = H->e_nuc;
    A.e0 = e0;
    A.pa = p_alpha;
    A.pb = p_beta;
    A.ha = la->hdiag;
    A.hb = lb->hdiag;
    A.Va = la->V64;
    A.sb = B->sb;
    A.Na = B->Na;
    A.Nb = B->Nb;
    A.batch = batch;
    A.m = m;
    A.log_pi = log_pi;
    A.ct = ct;
    A.ce = ce;
    A.cs = cs;
    A.zsum = zsum;
    A.w = w;
    A.adv = adv;
    A.grad = grad;
    A.part = lpart;
    A.bad = bad;
    k_nqs_loss<<<gl, kRedThreads, 0, s>>>(A);
    k_sum_partials<<<1, kRedThreads, 0, s>>>(lpart, (int)gl, 3, lsum);
    k_nqs_loss_final<<<1, 1, 0, s>>>(lsum, m, ct, ce, cs, loss);
    HQ_LAUNCH_CHECK();
    unsigned int hb = 0;
    HQ_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, s));
    HQ_CUDA(cudaStreamSynchronize(s));
    if (hb)
      return fail(HINQS_ERR_ARG, "hinqs_nqs_loss: %u basis or minibatch indices outside [0, N)", hb);
    return HINQS_OK;
  };
  const int rc = run();
  dfree(zpart, s);
  dfree(zsum, s);
  dfree(lpart, s);
  dfree(lsum, s);
  dfree(bad, s);
  return rc;
}
