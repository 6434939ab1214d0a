// K3/K4/K5-7 on CUDA cores: the sigma product sigma = H_B c of Step 3,
//   sigma = H_a C + C H_b^T + sum (pq|rs) E^a_pq C (E^b_rs)^T + E_nuc C,
// for C the N_a x N_b matrix of c (alpha index slow), FP64 or FP32.
//
// Split of the terms (s = self, i.e. the diagonal pseudo-links p = q in I):
//   k_sigma_rows  (one block per R alpha rows, output rows owned, plain stores)
//     diagonal       H_a(I,I) + H_b(J,J) + sum_{i in Ia, j in Ib} (ii|jj) + E_nuc
//     beta  links    sum_{Jb} H_b(Ib,Jb) C(Ia,Jb)            (rows staged in smem)
//     alpha-self x beta singles  sum_{b} s_b [sum_{i in Ia} (ii|rs_b)] C(Ia,Jb)
//     alpha links    sum_{Ja} H_a(Ia,Ja) C(Ja,Ib)            (coalesced row reads)
//   k_sigma_ab    (one block per alpha string Ja, scatter with atomics)
//     for each alpha single link Ja -> Ia (pair pq, sign s_a):
//       sigma(Ia,Ib) += s_a sum_rs (pq|rs) D(Ja,Ib;rs),
//       D(Ja,Ib;rs) = sum_{beta singles Ib->Jb with pair rs} s_b C(Ja,Jb)
//                     + [rs = jj, j in Ib] C(Ja,Ib)        (beta self)
#include <algorithm>

#include "hinqs_internal.cuh"

namespace hinqs {

template <typename T>
struct Prec;
template <>
struct Prec<double> {
  static const double* hval(const hinqs_links_s* L) { return L->hval64; }
  static const double* V(const hinqs_links_s* L) { return L->V64; }
  static const double* eri(const hinqs_ham_s* H) { return H->eri; }
};
template <>
struct Prec<float> {
  static const float* hval(const hinqs_links_s* L) { return L->hval32; }
  static const float* V(const hinqs_links_s* L) { return L->V32; }
  static const float* eri(const hinqs_ham_s* H) { return H->eri32; }
};

struct RowsArgs {
  int64_t Na, Nb;
  int n;
  double e_nuc;
  const int64_t* a_row;
  const int32_t* a_col;
  const int64_t* b_row;
  const int32_t* b_col;
  const int64_t* b_srow;
  const int2* b_slink;
  const double* a_hdiag;
  const double* b_hdiag;
  const uint64_t* sb;
};

// Same-spin parts, diagonal and alpha-self x beta-singles; R alpha rows per block.
// ROWS_SMEM: the R rows of C are staged in shared memory (else read from global).
template <typename T, int R, bool ROWS_SMEM>
__global__ void __launch_bounds__(256) k_sigma_rows(const T* __restrict__ C, T* __restrict__ sig,
                                                    RowsArgs A, const T* __restrict__ a_hval,
                                                    const T* __restrict__ b_hval,
                                                    const T* __restrict__ Va) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* VaS = reinterpret_cast<T*>(smem_raw);  // [R][n*n]
  const int n2 = A.n * A.n;
  T* Crow = VaS + R * n2;  // [R][Nb] when ROWS_SMEM
  const int64_t Ia0 = (int64_t)blockIdx.x * R;
  const int rows = (int)min64(R, A.Na - Ia0);
  for (int i = threadIdx.x; i < R * n2; i += blockDim.x) {
    int r = i / n2;
    VaS[i] = (r < rows) ? Va[(Ia0 + r) * n2 + (i % n2)] : T(0);
  }
  if (ROWS_SMEM) {
    for (int r = 0; r < R; ++r)
      for (int64_t j = threadIdx.x; j < A.Nb; j += blockDim.x)
        Crow[r * A.Nb + j] = (r < rows) ? C[(Ia0 + r) * A.Nb + j] : T(0);
  }
  __syncthreads();
  auto crow = [&](int r, int64_t j) -> T {
    if (ROWS_SMEM) return Crow[r * A.Nb + j];
    return (r < rows) ? C[(Ia0 + r) * A.Nb + j] : T(0);
  };
  double hda[R];
#pragma unroll
  for (int r = 0; r < R; ++r) hda[r] = (r < rows) ? A.a_hdiag[Ia0 + r] : 0.0;

  for (int64_t Ib = threadIdx.x; Ib < A.Nb; Ib += blockDim.x) {
    T acc[R];
    // diagonal
    const double hb = A.b_hdiag[Ib] + A.e_nuc;
    const uint64_t bits = A.sb[Ib];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T cross = T(0);
      uint64_t occ = bits;
      while (occ) {
        int j = __ffsll((long long)occ) - 1;
        occ &= occ - 1;
        cross += VaS[r * n2 + j * A.n + j];
      }
      T d = (T)(hda[r] + hb) + cross;
      acc[r] = d * crow(r, Ib);
    }
    // beta same-spin links
    for (int64_t k = A.b_row[Ib], e = A.b_row[Ib + 1]; k < e; ++k) {
      const int Jb = A.b_col[k];
      const T hv = b_hval[k];
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] += hv * crow(r, Jb);
    }
    // alpha self x beta singles
    for (int64_t k = A.b_srow[Ib], e = A.b_srow[Ib + 1]; k < e; ++k) {
      const int2 l = A.b_slink[k];
      const int sp = l.y;
      const int rs = (sp > 0 ? sp : -sp) - 1;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        T v = VaS[r * n2 + rs] * crow(r, l.x);
        acc[r] += (sp > 0) ? v : -v;
      }
    }
    // alpha same-spin links: coalesced reads of the linked rows
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r >= rows) break;
      const int64_t Ia = Ia0 + r;
      T a = acc[r];
      for (int64_t k = A.a_row[Ia], e = A.a_row[Ia + 1]; k < e; ++k)
        a += a_hval[k] * C[(int64_t)A.a_col[k] * A.Nb + Ib];
      sig[Ia * A.Nb + Ib] = a;
    }
  }
}

struct AbArgs {
  int64_t Na, Nb;
  int n;
  const int64_t* a_srow;
  const int2* a_slink;
  const int64_t* b_srow;
  const int2* b_slink;
  const uint64_t* sb;
};

// Opposite-spin part, one block per alpha string Ja; CH alpha single links of Ja
// are processed per pass with their (pq|.) rows in smem, transposed to [rs][a].
template <typename T, int CH, bool ROW_SMEM>
__global__ void __launch_bounds__(256) k_sigma_ab(const T* __restrict__ C, T* __restrict__ sig,
                                                  AbArgs A, const T* __restrict__ eri) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n2 = A.n * A.n;
  T* eriT = reinterpret_cast<T*>(smem_raw);  // [n2][CH]
  int* tgt = reinterpret_cast<int*>(eriT + (size_t)n2 * CH);
  T* Crow = reinterpret_cast<T*>(tgt + CH + (16 / sizeof(int)));  // [Nb]
  const int64_t Ja = blockIdx.x;
  const int64_t a_beg = A.a_srow[Ja], a_end = A.a_srow[Ja + 1];
  if (a_beg == a_end) return;
  const T* Cg = C + Ja * A.Nb;
  if (ROW_SMEM) {
    for (int64_t j = threadIdx.x; j < A.Nb; j += blockDim.x) Crow[j] = Cg[j];
  }
  const T* row = ROW_SMEM ? Crow : Cg;
  for (int64_t a0 = a_beg; a0 < a_end; a0 += CH) {
    const int cnt = (int)min64(CH, a_end - a0);
    __syncthreads();
    for (int i = threadIdx.x; i < n2 * CH; i += blockDim.x) {
      int xy = i / CH, a = i % CH;
      T v = T(0);
      if (a < cnt) {
        int sp = A.a_slink[a0 + a].y;
        int pq = (sp > 0 ? sp : -sp) - 1;
        v = eri[(int64_t)pq * n2 + xy];
        if (sp < 0) v = -v;
      }
      eriT[i] = v;
    }
    if (threadIdx.x < CH) tgt[threadIdx.x] = (threadIdx.x < cnt) ? A.a_slink[a0 + threadIdx.x].x : 0;
    __syncthreads();
    for (int64_t Ib = threadIdx.x; Ib < A.Nb; Ib += blockDim.x) {
      T e[CH];
#pragma unroll
      for (int a = 0; a < CH; ++a) e[a] = T(0);
      for (int64_t k = A.b_srow[Ib], kend = A.b_srow[Ib + 1]; k < kend; ++k) {
        const int2 l = A.b_slink[k];
        const int sp = l.y;
        const int rs = (sp > 0 ? sp : -sp) - 1;
        T v = row[l.x];
        if (sp < 0) v = -v;
        const T* er = eriT + rs * CH;
#pragma unroll
        for (int a = 0; a < CH; ++a) e[a] += v * er[a];
      }
      {
        const T v = row[Ib];
        uint64_t occ = A.sb[Ib];
        while (occ) {
          int j = __ffsll((long long)occ) - 1;
          occ &= occ - 1;
          const T* er = eriT + (j * A.n + j) * CH;
#pragma unroll
          for (int a = 0; a < CH; ++a) e[a] += v * er[a];
        }
      }
#pragma unroll
      for (int a = 0; a < CH; ++a)
        if (a < cnt) atomicAdd(sig + (int64_t)tgt[a] * A.Nb + Ib, e[a]);
    }
  }
}

template <typename T, int R>
static int launch_rows(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                       const hinqs_links_s* lb, const T* c, T* sig, cudaStream_t s,
                       size_t smem_limit) {
  RowsArgs A{B->Na,        B->Nb,       H->n,        H->e_nuc,  la->row_ptr,
             la->col,      lb->row_ptr, lb->col,     lb->srow_ptr, lb->slink,
             la->hdiag,    lb->hdiag,   B->sb};
  const int n2 = H->n * H->n;
  size_t base = (size_t)R * n2 * sizeof(T);
  size_t with_rows = base + (size_t)R * B->Nb * sizeof(T);
  unsigned grid = (unsigned)ceil_div(B->Na, R);
  if (with_rows <= smem_limit) {
    auto kern = k_sigma_rows<T, R, true>;
    HQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)with_rows));
    kern<<<grid, 256, with_rows, s>>>(c, sig, A, Prec<T>::hval(la), Prec<T>::hval(lb),
                                      Prec<T>::V(la));
  } else {
    auto kern = k_sigma_rows<T, R, false>;
    HQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)base));
    kern<<<grid, 256, base, s>>>(c, sig, A, Prec<T>::hval(la), Prec<T>::hval(lb),
                                 Prec<T>::V(la));
  }
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

template <typename T, int CH>
static int launch_ab(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                     const hinqs_links_s* lb, const T* c, T* sig, cudaStream_t s,
                     size_t smem_limit) {
  AbArgs A{B->Na, B->Nb, H->n, la->srow_ptr, la->slink, lb->srow_ptr, lb->slink, B->sb};
  const int n2 = H->n * H->n;
  size_t base = (size_t)n2 * CH * sizeof(T) + (CH + 4) * sizeof(int);
  base = (base + 15) & ~(size_t)15;
  size_t with_row = base + (size_t)B->Nb * sizeof(T);
  if (with_row <= smem_limit) {
    auto kern = k_sigma_ab<T, CH, true>;
    HQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)with_row));
    kern<<<(unsigned)B->Na, 256, with_row, s>>>(c, sig, A, Prec<T>::eri(H));
  } else {
    auto kern = k_sigma_ab<T, CH, false>;
    HQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)base));
    kern<<<(unsigned)B->Na, 256, base, s>>>(c, sig, A, Prec<T>::eri(H));
  }
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

template <typename T>
static int sigma_impl(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                      const hinqs_links_s* lb, const T* c, T* sig, cudaStream_t s) {
  const size_t limit = 200 * 1024;
  const int n2 = H->n * H->n;
  // largest row tile whose rows fit in shared memory
  auto fits = [&](int R) { return (size_t)R * (n2 + B->Nb) * sizeof(T) <= limit; };
  int rc;
  if (fits(8) && B->Na >= 8 * kNumSMs) rc = launch_rows<T, 8>(H, B, la, lb, c, sig, s, limit);
  else if (fits(4) && B->Na >= 4 * kNumSMs) rc = launch_rows<T, 4>(H, B, la, lb, c, sig, s, limit);
  else if (fits(2) && B->Na >= 2 * kNumSMs) rc = launch_rows<T, 2>(H, B, la, lb, c, sig, s, limit);
  else rc = launch_rows<T, 1>(H, B, la, lb, c, sig, s, limit);
  if (rc) return rc;
  if (la->nsingle == 0) return HINQS_OK;
  size_t ch16 = (size_t)n2 * 16 * sizeof(T) + B->Nb * sizeof(T) + 256;
  if (ch16 <= limit) return launch_ab<T, 16>(H, B, la, lb, c, sig, s, limit);
  return launch_ab<T, 8>(H, B, la, lb, c, sig, s, limit);
}

int sigma_launch(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                 const hinqs_links_s* lb, const void* c, void* sigma, int precision,
                 cudaStream_t s) {
  if (precision == HINQS_PREC_FP64)
    return sigma_impl<double>(H, B, la, lb, (const double*)c, (double*)sigma, s);
  if (precision == HINQS_PREC_FP32)
    return sigma_impl<float>(H, B, la, lb, (const float*)c, (float*)sigma, s);
  return fail(HINQS_ERR_ARG, "hinqs_sigma: unknown precision %d", precision);
}

// hdiag[I] = H_a(Ia,Ia) + H_b(Ib,Ib) + sum_{j in Ib} V_a[Ia][jj] + E_nuc
__global__ void k_diag(const double* __restrict__ ha, const double* __restrict__ hb,
                       const double* __restrict__ Va, const uint64_t* __restrict__ sb, int64_t Na,
                       int64_t Nb, int n, double e_nuc, double* __restrict__ out) {
  const int n2 = n * n;
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < Na * Nb;
       I += (int64_t)gridDim.x * blockDim.x) {
    int64_t ia = I / Nb, ib = I - ia * Nb;
    double d = ha[ia] + hb[ib] + e_nuc;
    uint64_t occ = sb[ib];
    while (occ) {
      int j = __ffsll((long long)occ) - 1;
      occ &= occ - 1;
      d += Va[ia * n2 + j * n + j];
    }
    out[I] = d;
  }
}

int diag_launch(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                const hinqs_links_s* lb, double* hdiag, cudaStream_t s) {
  int64_t N = B->Na * B->Nb;
  k_diag<<<(unsigned)std::min<int64_t>(ceil_div(N, 256), 16 * kNumSMs), 256, 0, s>>>(
      la->hdiag, lb->hdiag, la->V64, B->sb, B->Na, B->Nb, H->n, H->e_nuc, hdiag);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

int check_triplet(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                  const hinqs_links_s* lb, const char* who) {
  if (!H || !B || !la || !lb) return fail(HINQS_ERR_ARG, "%s: NULL handle", who);
  if (la->spin != 0 || lb->spin != 1)
    return fail(HINQS_ERR_ARG, "%s: la must be alpha links and lb beta links", who);
  if (la->N != B->Na || lb->N != B->Nb || la->strings != B->sa || lb->strings != B->sb)
    return fail(HINQS_ERR_ARG, "%s: links were built for another subspace", who);
  if (H->n != B->n || H->n_alpha != B->n_alpha || H->n_beta != B->n_beta)
    return fail(HINQS_ERR_ARG, "%s: Hamiltonian and subspace disagree on sizes", who);
  return HINQS_OK;
}

}  // namespace hinqs

using namespace hinqs;

extern "C" int hinqs_diag(const hinqs_ham* H, const hinqs_subspace* B, const hinqs_links* la,
                          const hinqs_links* lb, double* hdiag, void* stream) {
  HQ_TRY(check_triplet(H, B, la, lb, "hinqs_diag"));
  if (!hdiag) return fail(HINQS_ERR_ARG, "hinqs_diag: hdiag is NULL");
  return diag_launch(H, B, la, lb, hdiag, (cudaStream_t)stream);
}

extern "C" int hinqs_sigma(const hinqs_ham* H, const hinqs_subspace* B, const hinqs_links* la,
                           const hinqs_links* lb, const void* c, void* sigma, int precision,
                           void* stream) {
  HQ_TRY(check_triplet(H, B, la, lb, "hinqs_sigma"));
  if (!c || !sigma) return fail(HINQS_ERR_ARG, "hinqs_sigma: NULL vector");
  if (c == sigma) return fail(HINQS_ERR_ARG, "hinqs_sigma: c and sigma must not overlap");
  return sigma_launch(H, B, la, lb, c, sigma, precision, (cudaStream_t)stream);
}
