// Step 3 over the basis list itself: the projected Hamiltonian [H_B]_ij = <x_i|H|x_j>
// on a list of determinants x_i that lie in the product of the list's distinct
// alpha and beta strings.  The product supplies the strings, the same-spin links
// and the per-string tables; the list selects its determinants, so the operator is
// P H P with P the projector on the list, applied to vectors of the list's length.
//
// Layout: entries sorted by product position I = i_a * N_b + i_b (so by alpha
// string, then beta string), with a row index arow over the alpha strings: the
// entries of alpha string a are [arow[a], arow[a+1]) with ascending beta index.
//
// sigma (gather form, one warp per entry k = (I_a, I_b), no atomics, so results are
// reproducible run to run), sigma_k = sum_l <x_k|H|x_l> c_l over the list entries l:
//   diagonal        H_kk c_k
//   alpha links     J_a linked to I_a (singles, doubles) with J_b = I_b: the entry
//                   (J_a, I_b) is looked up in J_a's row by binary search; element =
//                   same-spin alpha element (+ alpha single x beta self term)
//   beta links      J_b linked to I_b with J_a = I_a: looked up in I_a's own row;
//                   element = same-spin beta element (+ alpha self x beta single term)
//   single x single J_a an alpha single of I_a, J_b a beta single of I_b:
//                   (pq|rs) s_a s_b; J_a's row is scanned with XOR/popcount (the
//                   beta string differs by one excitation) when it is short, else
//                   the beta singles of I_b are looked up in it.
#include <algorithm>

#include "hinqs_internal.cuh"
#include "slater.cuh"

namespace hinqs {

namespace {

using slater::find_string;
using slater::single_sign;

constexpr uint64_t kNoEntry = ~0ull;

__global__ void k_list_keys(const uint64_t* __restrict__ xa, const uint64_t* __restrict__ xb,
                            int64_t m, int64_t m_pad, const uint64_t* __restrict__ sa, int64_t Na,
                            const uint64_t* __restrict__ sb, int64_t Nb, uint64_t* __restrict__ keys,
                            unsigned int* bad) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m_pad;
       k += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = kNoEntry;
    if (k < m) {
      const int64_t a = find_string(sa, Na, xa[k]), b = find_string(sb, Nb, xb[k]);
      if (a < 0 || b < 0) atomicAdd(bad, 1u);
      else key = (uint64_t)(a * Nb + b);
    }
    keys[k] = key;
  }
}

__global__ void k_list_flags(const uint64_t* __restrict__ keys, int64_t m_pad, int64_t* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_pad;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (keys[i] != kNoEntry && (i == 0 || keys[i] != keys[i - 1])) ? 1 : 0;
}

__global__ void k_list_place(const uint64_t* __restrict__ keys, int64_t m_pad,
                             const int64_t* __restrict__ at, int64_t Nb, int64_t* __restrict__ pos,
                             int32_t* __restrict__ ia, int32_t* __restrict__ ib) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_pad;
       i += (int64_t)gridDim.x * blockDim.x)
    if (keys[i] != kNoEntry && (i == 0 || keys[i] != keys[i - 1])) {
      const int64_t I = (int64_t)keys[i], j = at[i];
      pos[j] = I;
      ia[j] = (int32_t)(I / Nb);
      ib[j] = (int32_t)(I % Nb);
    }
}

// arow[a] = first entry whose position is >= a * Nb (a = 0..Na)
__global__ void k_list_arow(const int64_t* __restrict__ pos, int64_t m, int64_t Na, int64_t Nb,
                            int64_t* __restrict__ arow) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a <= Na;
       a += (int64_t)gridDim.x * blockDim.x) {
    const int64_t key = a * Nb;
    int64_t lo = 0, hi = m;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (pos[mid] < key) lo = mid + 1;
      else hi = mid;
    }
    arow[a] = lo;
  }
}

// position of beta index b in the ascending ib[lo, hi), or -1
__device__ __forceinline__ int64_t find_in_row(const int32_t* __restrict__ ib, int64_t lo,
                                               int64_t hi, int32_t b) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    const int32_t v = __ldg(ib + mid);
    if (v == b) return mid;
    if (v < b) lo = mid + 1;
    else hi = mid;
  }
  return -1;
}

template <typename T>
struct ListArgs {
  int64_t m, Nb;
  int n;
  double e_nuc;
  const uint64_t* sa;
  const uint64_t* sb;
  const int32_t* ia;
  const int32_t* ib;
  const int64_t* arow;
  // alpha links
  const int64_t* a_rp;
  const int32_t* a_col;
  const T* a_hv;
  const uint32_t* a_exc;
  const int8_t* a_sign;
  const int8_t* a_deg;
  const int64_t* a_srp;
  const int2* a_sl;
  const T* a_V;  // [N_a][n^2] sum_{i in I_a} (ii|xy)
  const double* a_hd;
  const double* a_V64;
  // beta links
  const int64_t* b_rp;
  const int32_t* b_col;
  const T* b_hv;
  const uint32_t* b_exc;
  const int8_t* b_sign;
  const int8_t* b_deg;
  const int64_t* b_srp;
  const int2* b_sl;
  const T* b_V;
  const double* b_hd;
  const T* eri;  // (pq|rs) as [n^2][n^2]
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kListWarps = 8;

template <typename T>
__global__ void __launch_bounds__(32 * kListWarps) k_sigma_list(ListArgs<T> A,
                                                               const T* __restrict__ c,
                                                               T* __restrict__ sig) {
  const int lane = threadIdx.x & 31;
  const int n = A.n, n2 = n * n;
  for (int64_t k = (int64_t)blockIdx.x * kListWarps + (threadIdx.x >> 5); k < A.m;
       k += (int64_t)gridDim.x * kListWarps) {
    const int32_t a = A.ia[k], b = A.ib[k];
    const uint64_t Ib = A.sb[b];
    T acc = T(0);
    if (lane == 0) {  // diagonal: both same-spin diagonals, the (ii|jj) cross term, E_nuc
      double d = A.a_hd[a] + A.b_hd[b] + A.e_nuc;
      uint64_t o = Ib;
      while (o) {
        const int j = __ffsll((long long)o) - 1;
        o &= o - 1;
        d += A.a_V64[(int64_t)a * n2 + j * n + j];
      }
      acc = (T)d * c[k];
    }
    // alpha links of I_a with the beta string fixed
    for (int64_t e = A.a_rp[a] + lane; e < A.a_rp[a + 1]; e += 32) {
      const int32_t Ja = A.a_col[e];
      const int64_t l = find_in_row(A.ib, A.arow[Ja], A.arow[Ja + 1], b);
      if (l >= 0) {
        T el = A.a_hv[e];
        if (A.a_deg[e] == 1) {
          const uint32_t x = A.a_exc[e];
          el += (T)A.a_sign[e] * A.b_V[(int64_t)b * n2 + (int)(x & 255u) * n + (int)((x >> 8) & 255u)];
        }
        acc += el * c[l];
      }
    }
    // beta links of I_b with the alpha string fixed: look up in I_a's own row
    const int64_t r0 = A.arow[a], r1 = A.arow[a + 1];
    for (int64_t e = A.b_rp[b] + lane; e < A.b_rp[b + 1]; e += 32) {
      const int64_t l = find_in_row(A.ib, r0, r1, A.b_col[e]);
      if (l >= 0) {
        T el = A.b_hv[e];
        if (A.b_deg[e] == 1) {
          const uint32_t x = A.b_exc[e];
          el += (T)A.b_sign[e] * A.a_V[(int64_t)a * n2 + (int)(x & 255u) * n + (int)((x >> 8) & 255u)];
        }
        acc += el * c[l];
      }
    }
    // alpha single x beta single
    const int64_t bs0 = A.b_srp[b], bs1 = A.b_srp[b + 1];
    for (int64_t e = A.a_srp[a] + lane; e < A.a_srp[a + 1]; e += 32) {
      const int2 L = A.a_sl[e];
      const int pq = (L.y > 0 ? L.y : -L.y) - 1;
      const T sa_ = L.y > 0 ? T(1) : T(-1);
      const T* __restrict__ er = A.eri + (int64_t)pq * n2;
      const int64_t s0 = A.arow[L.x], s1 = A.arow[L.x + 1];
      if (s1 - s0 <= 2 * (bs1 - bs0) + 8) {
        for (int64_t l = s0; l < s1; ++l) {
          const uint64_t Jb = A.sb[A.ib[l]];
          const uint64_t x = Ib ^ Jb;
          if (__popcll(x) != 2) continue;
          const int r = __ffsll((long long)(Ib & x)) - 1;  // particle: in I_b, not J_b
          const int s = __ffsll((long long)(Jb & x)) - 1;  // hole: in J_b, not I_b
          const T v = er[r * n + s] * c[l];
          acc += (single_sign(Jb, r, s) > 0) == (sa_ > T(0)) ? v : -v;
        }
      } else {
        for (int64_t q = bs0; q < bs1; ++q) {
          const int2 Lb = A.b_sl[q];
          const int64_t l = find_in_row(A.ib, s0, s1, Lb.x);
          if (l < 0) continue;
          const T v = er[(Lb.y > 0 ? Lb.y : -Lb.y) - 1] * c[l];
          acc += (Lb.y > 0) == (sa_ > T(0)) ? v : -v;
        }
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) sig[k] = acc;
  }
}

__global__ void k_diag_list(const int32_t* __restrict__ ia, const int32_t* __restrict__ ib,
                            int64_t m, const double* __restrict__ ha, const double* __restrict__ hb,
                            const double* __restrict__ Va, const uint64_t* __restrict__ sb, int n,
                            double e_nuc, double* __restrict__ out) {
  const int n2 = n * n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = ia[k], b = ib[k];
    double d = ha[a] + hb[b] + e_nuc;
    uint64_t o = sb[b];
    while (o) {
      const int j = __ffsll((long long)o) - 1;
      o &= o - 1;
      d += Va[a * n2 + j * n + j];
    }
    out[k] = d;
  }
}

__global__ void k_list_scatter(const int64_t* __restrict__ pos, int64_t m,
                               const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x)
    y[pos[k]] = x[k];
}

__global__ void k_list_gather(const int64_t* __restrict__ pos, int64_t m,
                              const double* __restrict__ y, double* __restrict__ x) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x)
    x[k] = y[pos[k]];
}

template <typename T>
ListArgs<T> list_args(const hinqs_ham_s* H, const hinqs_links_s* la, const hinqs_links_s* lb,
                      const hinqs_detlist_s* L);
template <>
ListArgs<double> list_args<double>(const hinqs_ham_s* H, const hinqs_links_s* la,
                                   const hinqs_links_s* lb, const hinqs_detlist_s* L) {
  return ListArgs<double>{L->m, L->Nb, H->n, H->e_nuc, L->sa, L->sb, L->ia, L->ib, L->arow,
                          la->row_ptr, la->col, la->hval64, la->exc, la->sign, la->degree,
                          la->srow_ptr, la->slink, la->V64, la->hdiag, la->V64,
                          lb->row_ptr, lb->col, lb->hval64, lb->exc, lb->sign, lb->degree,
                          lb->srow_ptr, lb->slink, lb->V64, lb->hdiag, H->eri};
}
template <>
ListArgs<float> list_args<float>(const hinqs_ham_s* H, const hinqs_links_s* la,
                                 const hinqs_links_s* lb, const hinqs_detlist_s* L) {
  return ListArgs<float>{L->m, L->Nb, H->n, H->e_nuc, L->sa, L->sb, L->ia, L->ib, L->arow,
                         la->row_ptr, la->col, la->hval32, la->exc, la->sign, la->degree,
                         la->srow_ptr, la->slink, la->V32, la->hdiag, la->V64,
                         lb->row_ptr, lb->col, lb->hval32, lb->exc, lb->sign, lb->degree,
                         lb->srow_ptr, lb->slink, lb->V32, lb->hdiag, H->eri32};
}

unsigned list_grid(int64_t m, int per_block) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(m, per_block), 32 * kNumSMs));
}

}  // namespace

int check_list(const hinqs_subspace_s* B, const hinqs_detlist_s* L, const char* who) {
  if (!L) return fail(HINQS_ERR_ARG, "%s: NULL list", who);
  if (L->sa != B->sa || L->sb != B->sb || L->Na != B->Na || L->Nb != B->Nb)
    return fail(HINQS_ERR_ARG, "%s: the list was built on another subspace", who);
  return HINQS_OK;
}

int sigma_list_launch(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                      const hinqs_links_s* lb, const hinqs_detlist_s* L, const void* c,
                      void* sigma, int precision, cudaStream_t s) {
  (void)B;
  if (L->m == 0) return HINQS_OK;
  const unsigned grid = list_grid(L->m, kListWarps);
  if (precision == HINQS_PREC_FP64 || precision == HINQS_PREC_FP64_DFAB) {
    k_sigma_list<double><<<grid, 32 * kListWarps, 0, s>>>(list_args<double>(H, la, lb, L),
                                                           (const double*)c, (double*)sigma);
  } else if (precision >= HINQS_PREC_FP32 && precision <= HINQS_PREC_FP32_BF16C) {
    k_sigma_list<float><<<grid, 32 * kListWarps, 0, s>>>(list_args<float>(H, la, lb, L),
                                                          (const float*)c, (float*)sigma);
  } else {
    return fail(HINQS_ERR_ARG, "hinqs_sigma_list: unknown precision %d", precision);
  }
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

int diag_list_launch(const hinqs_ham_s* H, const hinqs_links_s* la, const hinqs_links_s* lb,
                     const hinqs_detlist_s* L, double* hdiag, cudaStream_t s) {
  if (L->m == 0) return HINQS_OK;
  k_diag_list<<<list_grid(L->m, 256), 256, 0, s>>>(L->ia, L->ib, L->m, la->hdiag, lb->hdiag,
                                                   la->V64, L->sb, H->n, H->e_nuc, hdiag);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

int check_triplet(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                  const hinqs_links_s* lb, const char* who);

}  // namespace hinqs

using namespace hinqs;

extern "C" int hinqs_detlist_create(const hinqs_subspace* B, const uint64_t* xa, const uint64_t* xb,
                                    int64_t m, hinqs_detlist** out, void* stream) {
  if (!out) return fail(HINQS_ERR_ARG, "hinqs_detlist_create: out is NULL");
  *out = nullptr;
  if (!B || m < 0 || (m > 0 && (!xa || !xb)))
    return fail(HINQS_ERR_ARG, "hinqs_detlist_create: NULL argument or negative size");
  if (B->Na > INT32_MAX || B->Nb > INT32_MAX)
    return fail(HINQS_ERR_ARG, "hinqs_detlist_create: more than 2^31 strings of one spin");
  cudaStream_t s = (cudaStream_t)stream;
  hinqs_detlist_s* L = new hinqs_detlist_s();
  L->Na = B->Na;
  L->Nb = B->Nb;
  L->sa = B->sa;
  L->sb = B->sb;
  int64_t m_pad = 2;
  while (m_pad < m) m_pad <<= 1;
  uint64_t* keys = nullptr;
  int64_t* at = nullptr;
  unsigned int* bad = nullptr;
  auto run = [&]() -> int {
    HQ_TRY(dalloc(&keys, m_pad, s));
    HQ_TRY(dalloc(&at, m_pad, s));
    HQ_TRY(dalloc(&bad, 1, s));
    HQ_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned int), s));
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(m_pad, 256), 16 * kNumSMs);
    k_list_keys<<<grid, 256, 0, s>>>(xa, xb, m, m_pad, B->sa, B->Na, B->sb, B->Nb, keys, bad);
    HQ_LAUNCH_CHECK();
    unsigned int hb = 0;
    HQ_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, s));
    HQ_CUDA(cudaStreamSynchronize(s));
    if (hb)
      return fail(HINQS_ERR_ARG, "hinqs_detlist_create: %u determinants are not in the product "
                                 "subspace", hb);
    HQ_TRY(bitonic_sort(keys, m_pad, s));
    k_list_flags<<<grid, 256, 0, s>>>(keys, m_pad, at);
    HQ_LAUNCH_CHECK();
    int64_t mu = 0;
    HQ_TRY(exclusive_scan_i64(at, at, m_pad, &mu, s));
    L->m = mu;
    HQ_TRY(dalloc(&L->pos, mu, s));
    HQ_TRY(dalloc(&L->ia, mu, s));
    HQ_TRY(dalloc(&L->ib, mu, s));
    HQ_TRY(dalloc(&L->arow, B->Na + 1, s));
    k_list_place<<<grid, 256, 0, s>>>(keys, m_pad, at, B->Nb, L->pos, L->ia, L->ib);
    k_list_arow<<<(unsigned)std::min<int64_t>(ceil_div(B->Na + 1, 256), 16 * kNumSMs), 256, 0, s>>>(
        L->pos, mu, B->Na, B->Nb, L->arow);
    HQ_LAUNCH_CHECK();
    return HINQS_OK;
  };
  const int rc = run();
  dfree(keys, s);
  dfree(at, s);
  dfree(bad, s);
  if (rc < 0) {
    hinqs_detlist_destroy(L);
    return rc;
  }
  *out = L;
  return HINQS_OK;
}

extern "C" int hinqs_detlist_size(const hinqs_detlist* L, int64_t* m) {
  if (!L || !m) return fail(HINQS_ERR_ARG, "hinqs_detlist_size: NULL argument");
  *m = L->m;
  return HINQS_OK;
}

extern "C" int hinqs_detlist_positions(const hinqs_detlist* L, int64_t* pos, void* stream) {
  if (!L || (L->m > 0 && !pos)) return fail(HINQS_ERR_ARG, "hinqs_detlist_positions: NULL argument");
  if (L->m == 0) return HINQS_OK;
  HQ_CUDA(cudaMemcpyAsync(pos, L->pos, L->m * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                          (cudaStream_t)stream));
  return HINQS_OK;
}

extern "C" int hinqs_detlist_destroy(hinqs_detlist* L) {
  if (!L) return HINQS_OK;
  cudaStream_t s = 0;
  cudaDeviceSynchronize();
  dfree(L->pos, s);
  dfree(L->ia, s);
  dfree(L->ib, s);
  dfree(L->arow, s);
  delete L;
  return HINQS_OK;
}

extern "C" int hinqs_detlist_scatter(const hinqs_detlist* L, const double* c_list,
                                     double* c_product, void* stream) {
  if (!L || (L->m > 0 && !c_list) || !c_product)
    return fail(HINQS_ERR_ARG, "hinqs_detlist_scatter: NULL argument");
  if (c_list == c_product) return fail(HINQS_ERR_ARG, "hinqs_detlist_scatter: vectors overlap");
  cudaStream_t s = (cudaStream_t)stream;
  HQ_CUDA(cudaMemsetAsync(c_product, 0, (size_t)(L->Na * L->Nb) * sizeof(double), s));
  if (L->m == 0) return HINQS_OK;
  k_list_scatter<<<list_grid(L->m, 256), 256, 0, s>>>(L->pos, L->m, c_list, c_product);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

extern "C" int hinqs_detlist_gather(const hinqs_detlist* L, const double* c_product,
                                    double* c_list, void* stream) {
  if (!L || !c_product || (L->m > 0 && !c_list))
    return fail(HINQS_ERR_ARG, "hinqs_detlist_gather: NULL argument");
  if (L->m == 0) return HINQS_OK;
  k_list_gather<<<list_grid(L->m, 256), 256, 0, (cudaStream_t)stream>>>(L->pos, L->m, c_product,
                                                                         c_list);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

extern "C" int hinqs_diag_list(const hinqs_ham* H, const hinqs_subspace* B, const hinqs_links* la,
                               const hinqs_links* lb, const hinqs_detlist* L, double* hdiag,
                               void* stream) {
  HQ_TRY(check_triplet(H, B, la, lb, "hinqs_diag_list"));
  HQ_TRY(check_list(B, L, "hinqs_diag_list"));
  if (L->m > 0 && !hdiag) return fail(HINQS_ERR_ARG, "hinqs_diag_list: hdiag is NULL");
  return diag_list_launch(H, la, lb, L, hdiag, (cudaStream_t)stream);
}

extern "C" int hinqs_sigma_list(const hinqs_ham* H, const hinqs_subspace* B, const hinqs_links* la,
                                const hinqs_links* lb, const hinqs_detlist* L, const void* c,
                                void* sigma, int precision, void* stream) {
  HQ_TRY(check_triplet(H, B, la, lb, "hinqs_sigma_list"));
  HQ_TRY(check_list(B, L, "hinqs_sigma_list"));
  if (L->m > 0 && (!c || !sigma)) return fail(HINQS_ERR_ARG, "hinqs_sigma_list: NULL vector");
  if (L->m > 0 && c == sigma)
    return fail(HINQS_ERR_ARG, "hinqs_sigma_list: c and sigma must not overlap");
  return sigma_list_launch(H, B, la, lb, L, c, sigma, precision, (cudaStream_t)stream);
}
