// K2: same-spin string links by XOR/popcount screening with warp ballots, their
// fermionic phases by masked popcount, and the same-spin Slater-Condon elements.
// Also the per-string tables used by the diagonal and the sigma.
#include <algorithm>

#include "hinqs_internal.cuh"

namespace hinqs {

__device__ __forceinline__ uint64_t below(int x) { return (1ull << x) - 1ull; }

__device__ __forceinline__ double eri_at(const double* __restrict__ eri, int n, int p, int q,
                                         int r, int s) {
  return eri[((int64_t)(p * n + q) * n + r) * n + s];
}

// Pass 1: one warp per row I counts the J with popcount(I^J) in {2,4} (all links)
// and == 2 (singles), scanning the sorted strings 32 at a time.
__global__ void k_links_count(const uint64_t* __restrict__ S, int64_t N, int64_t* cnt_all,
                              int64_t* cnt_single) {
  int lane = threadIdx.x & 31;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t I = warp; I < N; I += nwarps) {
    uint64_t x = S[I];
    int64_t ca = 0, cs = 0;
    for (int64_t j0 = 0; j0 < N; j0 += 32) {
      int64_t J = j0 + lane;
      int d = (J < N) ? __popcll(x ^ S[J]) : 0;
      unsigned ma = __ballot_sync(0xffffffffu, d == 2 || d == 4);
      unsigned ms = __ballot_sync(0xffffffffu, d == 2);
      ca += __popc(ma);
      cs += __popc(ms);
    }
    if (lane == 0) {
      cnt_all[I] = ca;
      cnt_single[I] = cs;
    }
  }
}

// Pass 2: the same scan writes the records in ascending J order; each hit's
// slot is its row offset plus the hits of lower lanes (ballot prefix count).
__global__ void k_links_fill(const uint64_t* __restrict__ S, int64_t N, int n,
                             const double* __restrict__ h, const double* __restrict__ eri,
                             const int64_t* __restrict__ row_ptr,
                             const int64_t* __restrict__ srow_ptr, int32_t* __restrict__ col,
                             double* __restrict__ hval64, float* __restrict__ hval32,
                             uint32_t* __restrict__ exc, int8_t* __restrict__ sign,
                             int8_t* __restrict__ degree, int2* __restrict__ slink) {
  int lane = threadIdx.x & 31;
  unsigned lt = (1u << lane) - 1u;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t I = warp; I < N; I += nwarps) {
    uint64_t x = S[I];
    int64_t pa = row_ptr[I], ps = srow_ptr[I];
    for (int64_t j0 = 0; j0 < N; j0 += 32) {
      int64_t J = j0 + lane;
      uint64_t y = (J < N) ? S[J] : x;
      uint64_t dx = x ^ y;
      int d = __popcll(dx);
      bool hit = (d == 2 || d == 4);
      unsigned ma = __ballot_sync(0xffffffffu, hit);
      unsigned ms = __ballot_sync(0xffffffffu, d == 2);
      if (hit) {
        int64_t slot = pa + __popc(ma & lt);
        uint64_t holes = x & dx, parts = y & dx;
        int q = __ffsll((long long)holes) - 1;
        int p = __ffsll((long long)parts) - 1;
        double v;
        int sg, r = 255, s = 255;
        if (d == 2) {
          // J = sign a+_p a_q I
          int n1 = __popcll(x & below(q));
          uint64_t x1 = x & ~(1ull << q);
          int n2 = __popcll(x1 & below(p));
          sg = ((n1 + n2) & 1) ? -1 : 1;
          double acc = h[p * n + q];
          uint64_t occ = x1;  // I without q
          while (occ) {
            int j = __ffsll((long long)occ) - 1;
            occ &= occ - 1;
            acc += eri_at(eri, n, p, q, j, j) - eri_at(eri, n, p, j, j, q);
          }
          v = sg * acc;
          int64_t sslot = ps + __popc(ms & lt);
          slink[sslot] = make_int2((int)J, sg * (p * n + q + 1));
        } else {
          // holes q < s, particles p < r: J = sign a+_p a+_r a_s a_q I
          s = 63 - __clzll((long long)holes);
          r = 63 - __clzll((long long)parts);
          int n1 = __popcll(x & below(q));
          uint64_t x1 = x & ~(1ull << q);
          int n2 = __popcll(x1 & below(s));
          uint64_t x2 = x1 & ~(1ull << s);
          int n3 = __popcll(x2 & below(r));
          uint64_t x3 = x2 | (1ull << r);
          int n4 = __popcll(x3 & below(p));
          sg = ((n1 + n2 + n3 + n4) & 1) ? -1 : 1;
          v = sg * (eri_at(eri, n, p, q, r, s) - eri_at(eri, n, p, s, r, q));
        }
        col[slot] = (int32_t)J;
        hval64[slot] = v;
        hval32[slot] = (float)v;
        exc[slot] = (uint32_t)p | ((uint32_t)q << 8) | ((uint32_t)r << 16) | ((uint32_t)s << 24);
        sign[slot] = (int8_t)sg;
        degree[slot] = (int8_t)(d / 2);
      }
      pa += __popc(ma);
      ps += __popc(ms);
    }
  }
}

// Per-string tables: hdiag[I] = sum_{i in I} h_ii + 1/2 sum_{i,j in I} [(ii|jj) - (ij|ji)],
// V[I][xy] = sum_{i in I} (ii|xy).  One block per string.
__global__ void k_string_tables(const uint64_t* __restrict__ S, int64_t N, int n,
                                const double* __restrict__ h, const double* __restrict__ eri,
                                double* __restrict__ hdiag, double* __restrict__ V64,
                                float* __restrict__ V32, double* __restrict__ VT64,
                                float* __restrict__ VT32, float* __restrict__ VTlo32) {
  int n2 = n * n;
  for (int64_t I = blockIdx.x; I < N; I += gridDim.x) {
    uint64_t x = S[I];
    for (int xy = threadIdx.x; xy < n2; xy += blockDim.x) {
      double acc = 0.0;
      uint64_t occ = x;
      while (occ) {
        int i = __ffsll((long long)occ) - 1;
        occ &= occ - 1;
        acc += eri[(int64_t)(i * n + i) * n2 + xy];
      }
      V64[I * n2 + xy] = acc;
      V32[I * n2 + xy] = (float)acc;
      VT64[(int64_t)xy * N + I] = acc;
      VT32[(int64_t)xy * N + I] = (float)acc;
      VTlo32[(int64_t)xy * N + I] = (float)(acc - (double)(float)acc);
    }
    if (threadIdx.x == 0) {
      double e1 = 0.0, e2 = 0.0;
      uint64_t oi = x;
      while (oi) {
        int i = __ffsll((long long)oi) - 1;
        oi &= oi - 1;
        e1 += h[i * n + i];
        uint64_t oj = x;
        while (oj) {
          int j = __ffsll((long long)oj) - 1;
          oj &= oj - 1;
          e2 += eri_at(eri, n, i, i, j, j) - eri_at(eri, n, i, j, j, i);
        }
      }
      hdiag[I] = e1 + 0.5 * e2;
    }
  }
}

// Slot-major copy of the single links plus the diagonal pseudo-links of each row,
// and the same slots with the pair replaced by its tensor-core operand offset.
__device__ __forceinline__ int tc_kpart(int pair, int n) {
  const int p = pair / n, q = pair % n;
  const int kf = p >= q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p;
  return (kf >> 3) * 128 + (kf & 7) * 2;
}

__global__ void k_build_ell(const uint64_t* __restrict__ S, int64_t N, int n,
                            const int64_t* __restrict__ srp, const int2* __restrict__ sl,
                            int width, int2* __restrict__ ell, int2* __restrict__ tcell,
                            uint32_t* __restrict__ tcq, int* __restrict__ cnt) {
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < N;
       I += (int64_t)gridDim.x * blockDim.x) {
    int k = 0;
    for (int64_t q = srp[I]; q < srp[I + 1]; ++q, ++k) {
      const int2 l = sl[q];
      ell[(int64_t)k * N + I] = l;
      const int kp = tc_kpart((l.y > 0 ? l.y : -l.y) - 1, n);
      tcell[(((int64_t)(k >> 1) * N + I) << 1) + (k & 1)] =
          make_int2(l.x, l.y > 0 ? kp : (int)((unsigned)kp | 0x80000000u));
      if (tcq)
        tcq[(((int64_t)(k >> 2) * N + I) << 2) + (k & 3)] =
            (uint32_t)l.x | ((uint32_t)kp << 17) | (l.y > 0 ? 0u : 0x80000000u);
    }
    uint64_t o = S[I];
    while (o) {
      int j = __ffsll((long long)o) - 1;
      o &= o - 1;
      ell[(int64_t)k * N + I] = make_int2((int)I, j * n + j + 1);
      tcell[(((int64_t)(k >> 1) * N + I) << 1) + (k & 1)] = make_int2((int)I, tc_kpart(j * n + j, n));
      if (tcq)
        tcq[(((int64_t)(k >> 2) * N + I) << 2) + (k & 3)] =
            (uint32_t)I | ((uint32_t)tc_kpart(j * n + j, n) << 17);
      ++k;
    }
    cnt[I] = k;
    for (; k < width; ++k) ell[(int64_t)k * N + I] = make_int2(0, 0);
    for (k = cnt[I]; k < ((width + 1) & ~1); ++k)
      tcell[(((int64_t)(k >> 1) * N + I) << 1) + (k & 1)] = make_int2(0, 0);
    if (tcq)
      for (k = cnt[I]; k < ((width + 3) & ~3); ++k) tcq[(((int64_t)(k >> 2) * N + I) << 2) + (k & 3)] = 0u;
  }
}

// Packed link records for the row products (see hinqs_links_s).
__global__ void k_pack_records(const int32_t* __restrict__ col, const double* __restrict__ h64,
                               int64_t nnz, int64_t other, int2* __restrict__ r32,
                               int4* __restrict__ r64, int64_t ld16, int2* __restrict__ r16) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t off = (uint32_t)((int64_t)col[k] * other);
    const double h = h64[k];
    r32[k] = make_int2((int)off, __float_as_int((float)h));
    const long long b = __double_as_longlong(h);
    r64[k] = make_int4((int)off, 0, (int)(b & 0xffffffffll), (int)(b >> 32));
    if (r16) r16[k] = make_int2((int)(uint32_t)((int64_t)col[k] * ld16), __float_as_int((float)h));
  }
}

// exc unpacking for export
__global__ void k_unpack_exc(const uint32_t* __restrict__ exc, int64_t nnz, uint8_t* p,
                             uint8_t* q, uint8_t* r, uint8_t* s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t e = exc[i];
    if (p) p[i] = (uint8_t)(e & 255u);
    if (q) q[i] = (uint8_t)((e >> 8) & 255u);
    if (r) r[i] = (uint8_t)((e >> 16) & 255u);
    if (s) s[i] = (uint8_t)(e >> 24);
  }
}

__global__ void k_row_max(const int64_t* __restrict__ rp, int64_t N, int* out) {
  int m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (int)(rp[i + 1] - rp[i]));
  atomicMax(out, m);
}

static void free_links(hinqs_links_s* L, cudaStream_t s) {
  dfree(L->row_ptr, s);
  dfree(L->col, s);
  dfree(L->hval64, s);
  dfree(L->hval32, s);
  dfree(L->exc, s);
  dfree(L->sign, s);
  dfree(L->degree, s);
  dfree(L->srow_ptr, s);
  dfree(L->slink, s);
  dfree(L->hdiag, s);
  dfree(L->V64, s);
  dfree(L->V32, s);
  dfree(L->VT64, s);
  dfree(L->VT32, s);
  dfree(L->VTlo32, s);
  dfree(L->sell, s);
  dfree(L->tcell, s);
  dfree(L->tcq, s);
  dfree(L->scount, s);
  dfree(L->rec32, s);
  dfree(L->rec64, s);
  dfree(L->rec16, s);
}

}  // namespace hinqs

using namespace hinqs;

extern "C" int hinqs_string_links(const hinqs_ham* H, const hinqs_subspace* B, int spin,
                                  hinqs_links** out, void* stream) {
  if (!out) return fail(HINQS_ERR_ARG, "hinqs_string_links: out is NULL");
  *out = nullptr;
  if (!H || !B) return fail(HINQS_ERR_ARG, "hinqs_string_links: NULL handle");
  if (spin != 0 && spin != 1) return fail(HINQS_ERR_ARG, "hinqs_string_links: spin must be 0 or 1");
  if (H->n != B->n || H->n_alpha != B->n_alpha || H->n_beta != B->n_beta)
    return fail(HINQS_ERR_ARG, "hinqs_string_links: Hamiltonian and subspace disagree on sizes");
  cudaStream_t s = (cudaStream_t)stream;
  hinqs_links_s* L = new hinqs_links_s();
  L->spin = spin;
  L->n = B->n;
  L->n_e = spin ? B->n_beta : B->n_alpha;
  L->N = spin ? B->Nb : B->Na;
  L->strings = spin ? B->sb : B->sa;
  const int64_t N = L->N;
  const int n = L->n, n2 = n * n;
  int64_t *ca = nullptr, *cs = nullptr;
  int* dmax = nullptr;
  int rc = HINQS_OK;
  auto cleanup = [&]() {
    dfree(ca, s);
    dfree(cs, s);
    dfree(dmax, s);
  };
  if ((rc = dalloc(&L->row_ptr, N + 1, s)) || (rc = dalloc(&L->srow_ptr, N + 1, s)) ||
      (rc = dalloc(&ca, N + 1, s)) || (rc = dalloc(&cs, N + 1, s)) || (rc = dalloc(&dmax, 2, s))) {
    cleanup();
    free_links(L, s);
    delete L;
    return rc;
  }
  int warps_per_block = 8;
  int grid = (int)std::min<int64_t>(ceil_div(N, warps_per_block), 16 * kNumSMs);
  k_links_count<<<grid, 32 * warps_per_block, 0, s>>>(L->strings, N, ca, cs);
  cudaMemsetAsync(ca + N, 0, sizeof(int64_t), s);
  cudaMemsetAsync(cs + N, 0, sizeof(int64_t), s);
  rc = exclusive_scan_i64(ca, L->row_ptr, N + 1, &L->nnz, s);
  if (!rc) rc = exclusive_scan_i64(cs, L->srow_ptr, N + 1, &L->nsingle, s);
  if (!rc) {
    if ((rc = dalloc(&L->col, L->nnz, s)) || (rc = dalloc(&L->hval64, L->nnz, s)) ||
        (rc = dalloc(&L->hval32, L->nnz, s)) || (rc = dalloc(&L->exc, L->nnz, s)) ||
        (rc = dalloc(&L->sign, L->nnz, s)) || (rc = dalloc(&L->degree, L->nnz, s)) ||
        (rc = dalloc(&L->slink, L->nsingle, s)) || (rc = dalloc(&L->hdiag, N, s)) ||
        (rc = dalloc(&L->V64, N * n2, s)) || (rc = dalloc(&L->V32, N * n2, s)) ||
        (rc = dalloc(&L->VT64, N * n2, s)) || (rc = dalloc(&L->VT32, N * n2, s)) ||
        (rc = dalloc(&L->VTlo32, N * n2, s))) {
    }
  }
  if (!rc) {
    k_links_fill<<<grid, 32 * warps_per_block, 0, s>>>(L->strings, N, n, H->h, H->eri, L->row_ptr,
                                                       L->srow_ptr, L->col, L->hval64, L->hval32,
                                                       L->exc, L->sign, L->degree, L->slink);
    k_string_tables<<<(unsigned)std::min<int64_t>(N, 16 * kNumSMs), 128, 0, s>>>(
        L->strings, N, n, H->h, H->eri, L->hdiag, L->V64, L->V32, L->VT64, L->VT32, L->VTlo32);
    cudaMemsetAsync(dmax, 0, 2 * sizeof(int), s);
    int g2 = (int)std::min<int64_t>(ceil_div(N, 256), 4 * kNumSMs);
    k_row_max<<<g2, 256, 0, s>>>(L->row_ptr, N, dmax);
    k_row_max<<<g2, 256, 0, s>>>(L->srow_ptr, N, dmax + 1);
    int hm[2] = {0, 0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hm, dmax, sizeof(hm), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "hinqs_string_links", __FILE__, __LINE__);
    L->max_row = hm[0];
    L->max_srow = hm[1];
  }
  if (!rc) {
    L->ell_width = L->max_srow + L->n_e;
    if (!(rc = dalloc(&L->sell, (size_t)std::max(1, L->ell_width) * N, s)) &&
        !(rc = dalloc(&L->tcell, (size_t)std::max(2, (L->ell_width + 1) & ~1) * N, s)) &&
        !(rc = dalloc(&L->scount, N, s)) &&
        !(N <= (int64_t(1) << 17) && n <= kTcMaxOrb &&
          (rc = dalloc(&L->tcq, (size_t)std::max(4, (L->ell_width + 3) & ~3) * N, s)))) {
      k_build_ell<<<(unsigned)std::min<int64_t>(ceil_div(N, 256), 4 * kNumSMs), 256, 0, s>>>(
          L->strings, N, n, L->srow_ptr, L->slink, L->ell_width, L->sell, L->tcell, L->tcq,
          L->scount);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) rc = cuda_fail(e, "k_build_ell", __FILE__, __LINE__);
    }
  }
  if (!rc && (uint64_t)B->Na * (uint64_t)B->Nb < (1ull << 32)) {
    const int64_t other = spin ? B->Na : B->Nb;
    const int64_t ld16 = (other + 63) / 64 * 64;
    const bool want16 = (uint64_t)N * (uint64_t)ld16 < (1ull << 32);
    if (!(rc = dalloc(&L->rec32, L->nnz, s)) && !(rc = dalloc(&L->rec64, L->nnz, s)) &&
        !(want16 && (rc = dalloc(&L->rec16, L->nnz, s)))) {
      L->ld16 = want16 ? ld16 : 0;
      k_pack_records<<<(unsigned)std::min<int64_t>(ceil_div(L->nnz, 256) + 1, 16 * kNumSMs), 256, 0,
                       s>>>(L->col, L->hval64, L->nnz, other, L->rec32, L->rec64, ld16, L->rec16);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) rc = cuda_fail(e, "k_pack_records", __FILE__, __LINE__);
    }
  }
  cleanup();
  if (rc) {
    free_links(L, s);
    delete L;
    return rc;
  }
  *out = L;
  return HINQS_OK;
}

extern "C" int hinqs_links_count(const hinqs_links* L, int64_t* n_links, int64_t* n_singles,
                                 int64_t* max_row) {
  if (!L) return fail(HINQS_ERR_ARG, "hinqs_links_count: NULL handle");
  if (n_links) *n_links = L->nnz;
  if (n_singles) *n_singles = L->nsingle;
  if (max_row) *max_row = L->max_row;
  return HINQS_OK;
}

extern "C" int hinqs_links_export(const hinqs_links* L, int64_t* row_ptr, int32_t* col,
                                  int8_t* degree, uint8_t* p, uint8_t* q, uint8_t* r, uint8_t* s,
                                  int8_t* sign, double* hval, void* stream) {
  if (!L) return fail(HINQS_ERR_ARG, "hinqs_links_export: NULL handle");
  cudaStream_t st = (cudaStream_t)stream;
  auto cp = [&](void* dst, const void* src, size_t bytes) -> int {
    if (dst && bytes) HQ_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
    return HINQS_OK;
  };
  HQ_TRY(cp(row_ptr, L->row_ptr, (L->N + 1) * sizeof(int64_t)));
  HQ_TRY(cp(col, L->col, L->nnz * sizeof(int32_t)));
  HQ_TRY(cp(degree, L->degree, L->nnz));
  HQ_TRY(cp(sign, L->sign, L->nnz));
  HQ_TRY(cp(hval, L->hval64, L->nnz * sizeof(double)));
  if ((p || q || r || s) && L->nnz) {
    k_unpack_exc<<<(unsigned)std::min<int64_t>(ceil_div(L->nnz, 256), 4 * kNumSMs), 256, 0, st>>>(
        L->exc, L->nnz, p, q, r, s);
    HQ_LAUNCH_CHECK();
  }
  return HINQS_OK;
}

extern "C" int hinqs_links_max_singles(const hinqs_links* L) { return L ? L->max_srow : 0; }

extern "C" int hinqs_links_tuning(const hinqs_links* L, int* rows_per_warp, int* chunk,
                                  int* stages) {
  if (!L) return fail(HINQS_ERR_ARG, "hinqs_links_tuning: NULL handle");
  if (rows_per_warp) *rows_per_warp = L->tune_rows;
  if (chunk) *chunk = L->tune_ch;
  if (stages) *stages = L->tune_stages;
  return HINQS_OK;
}

extern "C" int hinqs_links_set_tuning(hinqs_links* la, hinqs_links* lb, int rows_per_warp, int chunk,
                                      int stages) {
  if (!la || !lb || la->spin != 0 || lb->spin != 1)
    return fail(HINQS_ERR_ARG, "hinqs_links_set_tuning: la must be alpha links and lb beta links");
  if ((rows_per_warp != 0 && rows_per_warp != 2 && rows_per_warp != 4 && rows_per_warp != 8) ||
      (chunk != 0 && chunk != 8 && chunk != 16 && chunk != 32) || stages < 0 || stages > 3)
    return fail(HINQS_ERR_ARG, "hinqs_links_set_tuning: rows_per_warp in {0,2,4,8}, chunk in "
                               "{0,8,16,32}, stages in 0..3");
  la->tune_rows = lb->tune_rows = rows_per_warp;
  la->tune_ch = chunk;
  la->tune_stages = stages;
  return HINQS_OK;
}

extern "C" int hinqs_links_destroy(hinqs_links* L) {
  if (!L) return HINQS_OK;
  cudaDeviceSynchronize();
  free_links(L, 0);
  delete L;
  return HINQS_OK;
}
