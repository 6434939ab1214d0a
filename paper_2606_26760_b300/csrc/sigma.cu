// K3/K4/K5-7 on CUDA cores: the sigma product sigma = H_B c of Step 3,
//   sigma = H_a C + C H_b^T + sum (pq|rs) E^a_pq C (E^b_rs)^T + E_nuc C,
// for C the N_a x N_b matrix of c (alpha index slow), FP64 or FP32.
//
// Pipeline of one product (s = "self", the diagonal pseudo-links p = q in I):
//   CT = C^T                                   (tiled transpose)
//   ST = H_b CT + [alpha-self x beta singles]   (k_spmm_rows over beta rows, lane = alpha column)
//   sigma = ST^T                               (tiled transpose)
//   sigma += H_a C + diag * C                  (k_spmm_rows over alpha rows, lane = beta column)
//   sigma += opposite-spin singles x (singles + self)   (k_sigma_ab, scatter with atomics)
// The same-spin terms are sparse row products: a warp owns one output row, its 32
// lanes 32 consecutive columns, so every link record is a warp-uniform load and
// every operand load is a coalesced 128/256-byte row segment; 32 consecutive rows
// per block share most of their linked rows, which stay in L1.
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

template <typename T>
const T* VTof(const hinqs_links_s* L);
template <>
const double* VTof<double>(const hinqs_links_s* L) { return L->VT64; }
template <>
const float* VTof<float>(const hinqs_links_s* L) { return L->VT32; }

constexpr int kRowsPerWarp = 4;
constexpr int kRowWarps = 8;

// Y[I][c] = (accumulate ? Y[I][c] : 0)
//         + sum_{links k of row I} hv[k] * X[col[k]][c]
//         + sum_{singles k of row I} sign_k * VT[pair_k][c] * X[J_k][c]      (if srp)
//         + (hd_row[I] + hd_col[c] + e_nuc + sum_{j in scol[c]} Vrow[I][jj]) * X[I][c]  (if hd_row)
template <typename T>
__global__ void __launch_bounds__(256) k_spmm_rows(
    const T* __restrict__ X, T* __restrict__ Y, int64_t nrows, int64_t ncols,
    const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const T* __restrict__ hv,
    const int64_t* __restrict__ srp, const int2* __restrict__ sl, const T* __restrict__ VT,
    const double* __restrict__ hd_row, const double* __restrict__ hd_col, double e_nuc,
    const T* __restrict__ Vrow, const uint64_t* __restrict__ scol, int n, int accumulate) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c = (int64_t)blockIdx.x * 32 + lane;
  const bool active = c < ncols;
  const int64_t cc = active ? c : 0;
  const int n2 = n * n;
  const int64_t I0 = ((int64_t)blockIdx.y * kRowWarps + warp) * kRowsPerWarp;
  for (int rr = 0; rr < kRowsPerWarp; ++rr) {
    const int64_t I = I0 + rr;
    if (I >= nrows) break;
    T acc = (accumulate && active) ? Y[I * ncols + c] : T(0);
    if (hd_row) {
      // diagonal: the cross term sum_{j in scol[c]} Vrow[I][jj] by warp shuffles
      const T v0 = (lane < n) ? Vrow[I * n2 + lane * n + lane] : T(0);
      const T v1 = (lane + 32 < n) ? Vrow[I * n2 + (lane + 32) * n + lane + 32] : T(0);
      const uint64_t bits = scol[cc];
      T cross = T(0);
      for (int j = 0; j < n; ++j) {
        const T a = __shfl_sync(0xffffffffu, j < 32 ? v0 : v1, j & 31);
        if ((bits >> j) & 1ull) cross += a;
      }
      const T d = (T)(hd_row[I] + hd_col[cc] + e_nuc) + cross;
      if (active) acc += d * X[I * ncols + c];
    }
    int64_t k = rp[I];
    const int64_t e = rp[I + 1];
    for (; k + 4 <= e; k += 4) {
      const int j0 = col[k], j1 = col[k + 1], j2 = col[k + 2], j3 = col[k + 3];
      const T h0 = hv[k], h1 = hv[k + 1], h2 = hv[k + 2], h3 = hv[k + 3];
      const T x0 = X[(int64_t)j0 * ncols + cc], x1 = X[(int64_t)j1 * ncols + cc];
      const T x2 = X[(int64_t)j2 * ncols + cc], x3 = X[(int64_t)j3 * ncols + cc];
      acc += h0 * x0;
      acc += h1 * x1;
      acc += h2 * x2;
      acc += h3 * x3;
    }
    for (; k < e; ++k) acc += hv[k] * X[(int64_t)col[k] * ncols + cc];
    if (srp) {
      for (int64_t q = srp[I], qe = srp[I + 1]; q < qe; ++q) {
        const int2 l = sl[q];
        const int pair = (l.y > 0 ? l.y : -l.y) - 1;
        const T v = VT[(int64_t)pair * ncols + cc] * X[(int64_t)l.x * ncols + cc];
        acc += (l.y > 0) ? v : -v;
      }
    }
    if (active) Y[I * ncols + c] = acc;
  }
}

// out[j][i] = in[i][j] (+ out[j][i] if accumulate) for in of rows x cols; 32x32 tiles.
template <typename T>
__global__ void k_transpose_t(const T* __restrict__ in, T* __restrict__ out, int64_t rows,
                              int64_t cols, int accumulate) {
  __shared__ T tile[32][33];
  const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = by + k, j = bx + threadIdx.x;
    if (i < rows && j < cols) tile[k][threadIdx.x] = in[i * cols + j];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t j = bx + k, i = by + threadIdx.x;
    if (i < rows && j < cols) {
      T v = tile[threadIdx.x][k];
      if (accumulate) v += out[j * rows + i];
      out[j * rows + i] = v;
    }
  }
}

struct AbArgs {
  int64_t Na, Nb;
  int n;
  const int64_t* a_srow;
  const int2* a_slink;
  const int2* b_ell;   // slot-major beta singles + self, [width][Nb]
  const int* b_cnt;    // entries per beta string
};

// Opposite-spin part, one block per alpha string Ja.  CH alpha single links of Ja
// are processed per pass with their (pq|.) rows in shared memory, transposed to
// eriT[rs][a] with a padded row (no bank conflicts for the 16-byte loads of
// lanes that read different rs).  Each thread owns beta strings Ib and walks
// their single links and diagonal pseudo-links in slot-major order (coalesced).
template <typename T, int CH, bool ROW_SMEM>
__global__ void __launch_bounds__(256) k_sigma_ab(const T* __restrict__ C, T* __restrict__ sig,
                                                  AbArgs A, const T* __restrict__ eri) {
  constexpr int LD = CH + 16 / (int)sizeof(T);  // padded row of eriT
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n2 = A.n * A.n;
  T* eriT = reinterpret_cast<T*>(smem_raw);  // [n2][LD]
  int* tgt = reinterpret_cast<int*>(eriT + (size_t)n2 * LD);
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
      const int xy = i / CH, a = i % CH;
      T v = T(0);
      if (a < cnt) {
        const int sp = A.a_slink[a0 + a].y;
        const int pq = (sp > 0 ? sp : -sp) - 1;
        v = eri[(int64_t)pq * n2 + xy];
        if (sp < 0) v = -v;
      }
      eriT[xy * LD + a] = v;
    }
    if (threadIdx.x < CH) tgt[threadIdx.x] = (threadIdx.x < cnt) ? A.a_slink[a0 + threadIdx.x].x : 0;
    __syncthreads();
    for (int64_t Ib = threadIdx.x; Ib < A.Nb; Ib += blockDim.x) {
      T e[CH];
#pragma unroll
      for (int a = 0; a < CH; ++a) e[a] = T(0);
      const int nk = A.b_cnt[Ib];
      const int2* ell = A.b_ell + Ib;
      int k = 0;
      for (; k + 2 <= nk; k += 2) {
        const int2 l0 = ell[(int64_t)k * A.Nb], l1 = ell[(int64_t)(k + 1) * A.Nb];
        T v0 = row[l0.x], v1 = row[l1.x];
        if (l0.y < 0) v0 = -v0;
        if (l1.y < 0) v1 = -v1;
        const T* er0 = eriT + ((l0.y > 0 ? l0.y : -l0.y) - 1) * LD;
        const T* er1 = eriT + ((l1.y > 0 ? l1.y : -l1.y) - 1) * LD;
#pragma unroll
        for (int a = 0; a < CH; ++a) e[a] += v0 * er0[a] + v1 * er1[a];
      }
      if (k < nk) {
        const int2 l0 = ell[(int64_t)k * A.Nb];
        T v0 = row[l0.x];
        if (l0.y < 0) v0 = -v0;
        const T* er0 = eriT + ((l0.y > 0 ? l0.y : -l0.y) - 1) * LD;
#pragma unroll
        for (int a = 0; a < CH; ++a) e[a] += v0 * er0[a];
      }
#pragma unroll
      for (int a = 0; a < CH; ++a)
        if (a < cnt) atomicAdd(sig + (int64_t)tgt[a] * A.Nb + Ib, e[a]);
    }
  }
}

template <typename T, int CH>
static int launch_ab(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                     const hinqs_links_s* lb, const T* c, T* sig, cudaStream_t s,
                     size_t smem_limit) {
  AbArgs A{B->Na, B->Nb, H->n, la->srow_ptr, la->slink, lb->sell, lb->scount};
  const int n2 = H->n * H->n;
  constexpr int LD = CH + 16 / (int)sizeof(T);
  size_t base = (size_t)n2 * LD * sizeof(T) + (CH + 4) * sizeof(int);
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
static int transpose(const T* in, T* out, int64_t rows, int64_t cols, int accumulate,
                     cudaStream_t s) {
  dim3 tb(32, 8), tg((unsigned)ceil_div(cols, 32), (unsigned)ceil_div(rows, 32));
  k_transpose_t<T><<<tg, tb, 0, s>>>(in, out, rows, cols, accumulate);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

template <typename T>
static int spmm_rows(const T* X, T* Y, int64_t nrows, int64_t ncols, const hinqs_links_s* L,
                     const hinqs_links_s* Lsingles, const T* VT, const double* hd_row,
                     const double* hd_col, double e_nuc, const T* Vrow, const uint64_t* scol,
                     int n, int accumulate, cudaStream_t s) {
  dim3 grid((unsigned)ceil_div(ncols, 32), (unsigned)ceil_div(nrows, kRowWarps * kRowsPerWarp));
  k_spmm_rows<T><<<grid, 32 * kRowWarps, 0, s>>>(
      X, Y, nrows, ncols, L->row_ptr, L->col, Prec<T>::hval(L),
      Lsingles ? Lsingles->srow_ptr : nullptr, Lsingles ? Lsingles->slink : nullptr, VT, hd_row,
      hd_col, e_nuc, Vrow, scol, n, accumulate);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

template <typename T>
static int sigma_impl(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                      const hinqs_links_s* lb, const T* c, T* sig, cudaStream_t s,
                      int tc_split = 0) {
  const size_t limit = 200 * 1024;
  const int n = H->n, n2 = n * n;
  const int64_t Na = B->Na, Nb = B->Nb, N = Na * Nb;
  T *CT = nullptr, *ST = nullptr;
  int rc = HINQS_OK;
  if ((rc = dalloc(&CT, N, s)) || (rc = dalloc(&ST, N, s))) {
    dfree(CT, s);
    dfree(ST, s);
    return rc;
  }
  auto run = [&]() -> int {
    HQ_TRY(transpose<T>(c, CT, Na, Nb, 0, s));
    // beta same-spin links and alpha-self x beta singles, rows = beta strings
    HQ_TRY(spmm_rows<T>(CT, ST, Nb, Na, lb, lb, VTof<T>(la), nullptr, nullptr, 0.0, nullptr,
                        nullptr, n, 0, s));
    HQ_TRY(transpose<T>(ST, sig, Nb, Na, 0, s));
    // alpha same-spin links and the diagonal, rows = alpha strings
    HQ_TRY(spmm_rows<T>(c, sig, Na, Nb, la, nullptr, nullptr, la->hdiag, lb->hdiag, H->e_nuc,
                        Prec<T>::V(la), B->sb, n, 1, s));
    if (la->nsingle == 0) return HINQS_OK;
    if constexpr (sizeof(T) == 4) {
      if (tc_split) return sigma_ab_tc_launch(H, B, la, lb, c, sig, tc_split, s);
    }
    auto need = [&](int ch) { return (size_t)n2 * (ch + 16 / sizeof(T)) * sizeof(T) + 256; };
    if (sizeof(T) == 4 && need(32) <= limit / 2) return launch_ab<T, 32>(H, B, la, lb, c, sig, s, limit);
    if (need(16) <= limit / 2) return launch_ab<T, 16>(H, B, la, lb, c, sig, s, limit);
    return launch_ab<T, 8>(H, B, la, lb, c, sig, s, limit);
  };
  rc = run();
  dfree(CT, s);
  dfree(ST, s);
  return rc;
}

int sigma_launch(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                 const hinqs_links_s* lb, const void* c, void* sigma, int precision,
                 cudaStream_t s) {
  if (precision == HINQS_PREC_FP64)
    return sigma_impl<double>(H, B, la, lb, (const double*)c, (double*)sigma, s);
  if (precision == HINQS_PREC_FP32)
    return sigma_impl<float>(H, B, la, lb, (const float*)c, (float*)sigma, s);
  if (precision == HINQS_PREC_FP32_BF16AB)
    return sigma_impl<float>(H, B, la, lb, (const float*)c, (float*)sigma, s, 1);
  if (precision == HINQS_PREC_FP32_BF16X3AB)
    return sigma_impl<float>(H, B, la, lb, (const float*)c, (float*)sigma, s, 3);
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
  HQ_TRY(sigma_launch(H, B, la, lb, c, sigma, precision, (cudaStream_t)stream));
  if (precision == HINQS_PREC_FP32_BF16AB || precision == HINQS_PREC_FP32_BF16X3AB)
    return tc_error_check((cudaStream_t)stream);
  return HINQS_OK;
}
