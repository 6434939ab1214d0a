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
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

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

// Packed link records: {element offset of the linked row, element}.
template <typename T>
struct Rec;
template <>
struct Rec<float> {
  using type = int2;
  using vec2 = float2;
  __device__ static float h(const int2& r) { return __int_as_float(r.y); }
  __device__ static uint32_t off(const int2& r) { return (uint32_t)r.x; }
};
template <>
struct Rec<double> {
  using type = int4;
  using vec2 = double2;
  __device__ static double h(const int4& r) { return __hiloint2double(r.w, r.z); }
  __device__ static uint32_t off(const int4& r) { return (uint32_t)r.x; }
};

// Same row product as k_spmm_rows with packed records (no per-link index
// arithmetic), 8 links in flight per lane, and VEC consecutive columns per lane.
template <typename T, int VEC, int RPW>
__global__ void __launch_bounds__(256) k_spmm_rec(
    const T* __restrict__ X, T* __restrict__ Y, int64_t nrows, int64_t ncols,
    const int64_t* __restrict__ rp, const typename Rec<T>::type* __restrict__ rec,
    const int64_t* __restrict__ srp, const int2* __restrict__ sl, const T* __restrict__ VT,
    const double* __restrict__ hd_row, const double* __restrict__ hd_col, double e_nuc,
    const T* __restrict__ Vrow, const uint64_t* __restrict__ scol, int n, int accumulate) {
  using R = Rec<T>;
  using RT = typename R::type;
  using V2 = typename R::vec2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = ((int64_t)blockIdx.x * 32 + lane) * VEC;
  const bool active = c0 < ncols;  // VEC divides ncols
  const int64_t cc = active ? c0 : 0;
  const int n2 = n * n;
  const int64_t I0 = ((int64_t)blockIdx.y * kRowWarps + warp) * RPW;
  for (int rr = 0; rr < RPW; ++rr) {
    const int64_t I = I0 + rr;
    if (I >= nrows) break;
    T acc[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = (accumulate && active) ? Y[I * ncols + c0 + v] : T(0);
    if (hd_row) {
      const T v0 = (lane < n) ? Vrow[I * n2 + lane * n + lane] : T(0);
      const T v1 = (lane + 32 < n) ? Vrow[I * n2 + (lane + 32) * n + lane + 32] : T(0);
      uint64_t bits[VEC];
      T cross[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        bits[v] = scol[cc + v];
        cross[v] = T(0);
      }
      for (int j = 0; j < n; ++j) {
        const T a = __shfl_sync(0xffffffffu, j < 32 ? v0 : v1, j & 31);
#pragma unroll
        for (int v = 0; v < VEC; ++v)
          if ((bits[v] >> j) & 1ull) cross[v] += a;
      }
      if (active) {
#pragma unroll
        for (int v = 0; v < VEC; ++v)
          acc[v] += ((T)(hd_row[I] + hd_col[c0 + v] + e_nuc) + cross[v]) * X[I * ncols + c0 + v];
      }
    }
    const RT* __restrict__ r = rec + rp[I];
    const int nk = (int)(rp[I + 1] - rp[I]);
    const T* __restrict__ Xc = X + cc;
    int k = 0;
    for (; k + 8 <= nk; k += 8) {
      RT q[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) q[u] = r[k + u];
      if constexpr (VEC == 1) {
        T x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = Xc[R::off(q[u])];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[0] += R::h(q[u]) * x[u];
      } else {
        V2 x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = *reinterpret_cast<const V2*>(Xc + R::off(q[u]));
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          acc[0] += R::h(q[u]) * x[u].x;
          acc[1] += R::h(q[u]) * x[u].y;
        }
      }
    }
    for (; k < nk; ++k) {
      const RT q = r[k];
      if constexpr (VEC == 1) {
        acc[0] += R::h(q) * Xc[R::off(q)];
      } else {
        const V2 x = *reinterpret_cast<const V2*>(Xc + R::off(q));
        acc[0] += R::h(q) * x.x;
        acc[1] += R::h(q) * x.y;
      }
    }
    if (srp) {
      for (int64_t q = srp[I], qe = srp[I + 1]; q < qe; ++q) {
        const int2 l = sl[q];
        const int pair = (l.y > 0 ? l.y : -l.y) - 1;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const T t = VT[(int64_t)pair * ncols + cc + v] * X[(int64_t)l.x * ncols + cc + v];
          acc[v] += (l.y > 0) ? t : -t;
        }
      }
    }
    if (active) {
#pragma unroll
      for (int v = 0; v < VEC; ++v) Y[I * ncols + c0 + v] = acc[v];
    }
  }
}

// FP32 row product with four consecutive columns per lane (one 16-byte operand load
// per link and lane) and the link records of a row read 32 at a time by the whole
// warp (one coalesced 256-byte load) and broadcast by shuffles: per link, the L1 data
// path moves the 512-byte operand segment and 1/32 of a record line, instead of a
// 256-byte segment plus a warp-uniform record load.  Requires ncols % 4 == 0.
// four consecutive columns from p: one 16-byte load when the rows are 16-byte aligned
// (the column count a multiple of 4), else up to `nv` guarded scalar loads
template <bool ALIGNED>
__device__ __forceinline__ float4 ld4(const float* __restrict__ p, int nv) {
  if (ALIGNED) return __ldg(reinterpret_cast<const float4*>(p));
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (nv > 0) v.x = __ldg(p);
  if (nv > 1) v.y = __ldg(p + 1);
  if (nv > 2) v.z = __ldg(p + 2);
  if (nv > 3) v.w = __ldg(p + 3);
  return v;
}

template <int RPW, bool ALIGNED>
__device__ __forceinline__ void spmm_rec4_block(
    const float* __restrict__ X, float* __restrict__ Y, int64_t nrows, int64_t ncols,
    const int64_t* __restrict__ rp, const int2* __restrict__ rec,
    const int64_t* __restrict__ srp, const int2* __restrict__ sl, const float* __restrict__ VT,
    const double* __restrict__ hd_row, const double* __restrict__ hd_col, double e_nuc,
    const float* __restrict__ Vrow, const uint64_t* __restrict__ scol, int n, int accumulate,
    int64_t bx, int64_t by) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = (bx * 32 + lane) * 4;
  const bool active = c0 < ncols;
  const int64_t cc = active ? c0 : 0;
  const int nv = active ? (int)min64(4, ncols - c0) : 0;  // columns of this lane
  const int n2 = n * n;
  const unsigned full = 0xffffffffu;
  const int64_t I0 = (by * kRowWarps + warp) * RPW;
  for (int rr = 0; rr < RPW; ++rr) {
    const int64_t I = I0 + rr;
    if (I >= nrows) break;  // warp-uniform
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (accumulate && active) acc = ld4<ALIGNED>(Y + I * ncols + c0, nv);
    if (hd_row) {
      const float v0 = (lane < n) ? Vrow[I * n2 + lane * n + lane] : 0.f;
      const float v1 = (lane + 32 < n) ? Vrow[I * n2 + (lane + 32) * n + lane + 32] : 0.f;
      const uint64_t b0 = nv > 0 ? scol[cc] : 0, b1 = nv > 1 ? scol[cc + 1] : 0;
      const uint64_t b2 = nv > 2 ? scol[cc + 2] : 0, b3 = nv > 3 ? scol[cc + 3] : 0;
      float x0 = 0.f, x1 = 0.f, x2 = 0.f, x3 = 0.f;
      for (int j = 0; j < n; ++j) {
        const float a = __shfl_sync(full, j < 32 ? v0 : v1, j & 31);
        if ((b0 >> j) & 1ull) x0 += a;
        if ((b1 >> j) & 1ull) x1 += a;
        if ((b2 >> j) & 1ull) x2 += a;
        if ((b3 >> j) & 1ull) x3 += a;
      }
      if (active) {
        const float4 x = ld4<ALIGNED>(X + I * ncols + c0, nv);
        const double hr = hd_row[I] + e_nuc;
        acc.x += ((float)(hr + hd_col[c0]) + x0) * x.x;
        if (nv > 1) acc.y += ((float)(hr + hd_col[c0 + 1]) + x1) * x.y;
        if (nv > 2) acc.z += ((float)(hr + hd_col[c0 + 2]) + x2) * x.z;
        if (nv > 3) acc.w += ((float)(hr + hd_col[c0 + 3]) + x3) * x.w;
      }
    }
    const int2* __restrict__ r = rec + rp[I];
    const int nk = (int)(rp[I + 1] - rp[I]);
    const float* __restrict__ Xc = X + cc;
    for (int k0 = 0; k0 < nk; k0 += 32) {
      const int2 mine = (k0 + lane < nk) ? __ldg(r + k0 + lane) : make_int2(0, 0);
      const int cnt = min(32, nk - k0);
      int u = 0;
      for (; u + 8 <= cnt; u += 8) {
        float4 x[8];
        float h[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          const uint32_t off = (uint32_t)__shfl_sync(full, mine.x, u + v);
          h[v] = __int_as_float(__shfl_sync(full, mine.y, u + v));
          x[v] = ld4<ALIGNED>(Xc + off, nv);
        }
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          acc.x = fmaf(h[v], x[v].x, acc.x);
          acc.y = fmaf(h[v], x[v].y, acc.y);
          acc.z = fmaf(h[v], x[v].z, acc.z);
          acc.w = fmaf(h[v], x[v].w, acc.w);
        }
      }
      for (; u < cnt; ++u) {
        const uint32_t off = (uint32_t)__shfl_sync(full, mine.x, u);
        const float h = __int_as_float(__shfl_sync(full, mine.y, u));
        const float4 x = ld4<ALIGNED>(Xc + off, nv);
        acc.x = fmaf(h, x.x, acc.x);
        acc.y = fmaf(h, x.y, acc.y);
        acc.z = fmaf(h, x.z, acc.z);
        acc.w = fmaf(h, x.w, acc.w);
      }
    }
    if (srp && active) {
      for (int64_t q = srp[I], qe = srp[I + 1]; q < qe; ++q) {
        const int2 l = sl[q];
        const int pair = (l.y > 0 ? l.y : -l.y) - 1;
        const float4 vt = ld4<ALIGNED>(VT + (int64_t)pair * ncols + c0, nv);
        const float4 x = ld4<ALIGNED>(X + (int64_t)l.x * ncols + c0, nv);
        const float sg = l.y > 0 ? 1.f : -1.f;
        acc.x += sg * vt.x * x.x;
        acc.y += sg * vt.y * x.y;
        acc.z += sg * vt.z * x.z;
        acc.w += sg * vt.w * x.w;
      }
    }
    if (active) {
      float* y = Y + I * ncols + c0;
      if (ALIGNED) {
        *reinterpret_cast<float4*>(y) = acc;
      } else {
        y[0] = acc.x;
        if (nv > 1) y[1] = acc.y;
        if (nv > 2) y[2] = acc.z;
        if (nv > 3) y[3] = acc.w;
      }
    }
  }
}

template <int RPW>
__global__ void __launch_bounds__(256, 4) k_spmm_rec4(
    const float* __restrict__ X, float* __restrict__ Y, int64_t nrows, int64_t ncols,
    const int64_t* __restrict__ rp, const int2* __restrict__ rec,
    const int64_t* __restrict__ srp, const int2* __restrict__ sl, const float* __restrict__ VT,
    const double* __restrict__ hd_row, const double* __restrict__ hd_col, double e_nuc,
    const float* __restrict__ Vrow, const uint64_t* __restrict__ scol, int n, int accumulate) {
  spmm_rec4_block<RPW, true>(X, Y, nrows, ncols, rp, rec, srp, sl, VT, hd_row, hd_col, e_nuc, Vrow,
                             scol, n, accumulate, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// HINQS_PREC_FP32_BF16C: the same-spin row products read a BF16 copy of C (rounded
// once per product) with rows padded to 128 bytes, so a link moves half the bytes of
// the FP32 form and no operand segment straddles an extra line; products and sums in
// FP32, the diagonal term on the FP32 C.

// C (rows x cols, FP32) -> Cb (rows x ldc, BF16, round to nearest even) and its
// transpose CTb (cols x ldr, BF16); the padding columns of both are zero.  The grid
// covers ldc columns and ldr rows in 32 x 32 tiles.
__global__ void k_bf16_pack(const float* __restrict__ C, int64_t rows, int64_t cols,
                            __nv_bfloat16* __restrict__ Cb, int64_t ldc,
                            __nv_bfloat16* __restrict__ CTb, int64_t ldr) {
  __shared__ float tile[32][33];
  const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = by + k, j = bx + threadIdx.x;
    const float v = (i < rows && j < cols) ? C[i * cols + j] : 0.f;
    tile[k][threadIdx.x] = v;
    if (i < rows && j < ldc) Cb[i * ldc + j] = __float2bfloat16_rn(v);
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t j = bx + k, i = by + threadIdx.x;
    if (j < cols && i < ldr) CTb[j * ldr + i] = __float2bfloat16_rn(tile[threadIdx.x][k]);
  }
}

// eight consecutive FP32 values from p (nv of them valid): two 16-byte loads when the
// rows are 16-byte aligned (then nv is 4 or 8), else guarded scalar loads
template <bool ALIGNED>
__device__ __forceinline__ void ld8(const float* __restrict__ p, int nv, float* v) {
  if (ALIGNED) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    const float4 b = nv > 4 ? __ldg(reinterpret_cast<const float4*>(p + 4))
                            : make_float4(0.f, 0.f, 0.f, 0.f);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = i < nv ? __ldg(p + i) : 0.f;
  }
}

template <bool ALIGNED>
__device__ __forceinline__ void st8(float* __restrict__ p, int nv, const float* v) {
  if (ALIGNED) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    if (nv > 4) *reinterpret_cast<float4*>(p + 4) = make_float4(v[4], v[5], v[6], v[7]);
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (i < nv) p[i] = v[i];
  }
}

// acc[0..7] += h * (eight BF16 values packed in x); BF16 -> FP32 is a 16-bit shift
__device__ __forceinline__ void fma_bf16x8(float h, const uint4& x, float* acc) {
  const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    acc[2 * i] = fmaf(h, __uint_as_float(w[i] << 16), acc[2 * i]);
    acc[2 * i + 1] = fmaf(h, __uint_as_float(w[i] & 0xffff0000u), acc[2 * i + 1]);
  }
}

// The row product of k_spmm_rec4 on the BF16 operand: eight columns per lane (one
// 16-byte load per link and lane, a 512-byte segment of a 128-byte aligned row per
// warp), records {J * ldx, h} read 32 at a time and broadcast by shuffles.  X32 is
// the FP32 C for the diagonal term (alpha rows only); VT rows are FP32.  MODE 2 adds
// the diagonal term (alpha rows), 1 the alpha-self x beta-single term (beta rows), 0
// neither; without the diagonal's registers four blocks fit on an SM.
template <int RPW, bool ALIGNED, int MODE>
__device__ __forceinline__ void spmm_bf16_block(
    const __nv_bfloat16* __restrict__ Xb, int64_t ldx, const float* __restrict__ X32,
    float* __restrict__ Y, int64_t nrows, int64_t ncols, const int64_t* __restrict__ rp,
    const int2* __restrict__ rec, const int64_t* __restrict__ srp, const int2* __restrict__ sl,
    const float* __restrict__ VT, const double* __restrict__ hd_row,
    const double* __restrict__ hd_col, double e_nuc, const float* __restrict__ Vrow,
    const uint64_t* __restrict__ scol, int n, int accumulate, int64_t bx, int64_t by) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = (bx * 32 + lane) * 8;
  const bool active = c0 < ncols;
  const int64_t cc = active ? c0 : 0;
  const int nv = active ? (int)min64(8, ncols - c0) : 0;  // columns of this lane
  const int n2 = n * n;
  const unsigned full = 0xffffffffu;
  const int64_t I0 = (by * kRowWarps + warp) * RPW;
  for (int rr = 0; rr < RPW; ++rr) {
    const int64_t I = I0 + rr;
    if (I >= nrows) break;  // warp-uniform
    float acc[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[v] = 0.f;
    if (accumulate && active) ld8<ALIGNED>(Y + I * ncols + c0, nv, acc);
    if constexpr (MODE == 2) {
      const float v0 = (lane < n) ? Vrow[I * n2 + lane * n + lane] : 0.f;
      const float v1 = (lane + 32 < n) ? Vrow[I * n2 + (lane + 32) * n + lane + 32] : 0.f;
      uint64_t b[8];
      float xs[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) b[v] = v < nv ? scol[cc + v] : 0, xs[v] = 0.f;
      for (int j = 0; j < n; ++j) {
        const float a = __shfl_sync(full, j < 32 ? v0 : v1, j & 31);
#pragma unroll
        for (int v = 0; v < 8; ++v)
          if ((b[v] >> j) & 1ull) xs[v] += a;
      }
      if (active) {
        float x[8];
        ld8<ALIGNED>(X32 + I * ncols + c0, nv, x);
        const double hr = hd_row[I] + e_nuc;
#pragma unroll
        for (int v = 0; v < 8; ++v)
          if (v < nv) acc[v] += ((float)(hr + hd_col[c0 + v]) + xs[v]) * x[v];
      }
    }
    const int2* __restrict__ r = rec + rp[I];
    const int nk = (int)(rp[I + 1] - rp[I]);
    const __nv_bfloat16* __restrict__ Xc = Xb + cc;
    for (int k0 = 0; k0 < nk; k0 += 32) {
      const int2 mine = (k0 + lane < nk) ? __ldg(r + k0 + lane) : make_int2(0, 0);
      const int cnt = min(32, nk - k0);
      int u = 0;
      for (; u + 8 <= cnt; u += 8) {
        uint4 x[8];
        float h[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          const uint32_t off = (uint32_t)__shfl_sync(full, mine.x, u + v);
          h[v] = __int_as_float(__shfl_sync(full, mine.y, u + v));
          x[v] = __ldg(reinterpret_cast<const uint4*>(Xc + off));
        }
#pragma unroll
        for (int v = 0; v < 8; ++v) fma_bf16x8(h[v], x[v], acc);
      }
      for (; u < cnt; ++u) {
        const uint32_t off = (uint32_t)__shfl_sync(full, mine.x, u);
        const float h = __int_as_float(__shfl_sync(full, mine.y, u));
        fma_bf16x8(h, __ldg(reinterpret_cast<const uint4*>(Xc + off)), acc);
      }
    }
    if (MODE == 1 && active) {
      for (int64_t q = srp[I], qe = srp[I + 1]; q < qe; ++q) {
        const int2 l = sl[q];
        const int pair = (l.y > 0 ? l.y : -l.y) - 1;
        float vt[8], t[8];
        ld8<ALIGNED>(VT + (int64_t)pair * ncols + c0, nv, vt);
#pragma unroll
        for (int v = 0; v < 8; ++v) t[v] = 0.f;
        fma_bf16x8(1.f, __ldg(reinterpret_cast<const uint4*>(Xb + (int64_t)l.x * ldx + c0)), t);
        const float sg = l.y > 0 ? 1.f : -1.f;
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[v] += sg * vt[v] * t[v];
      }
    }
    if (active) st8<ALIGNED>(Y + I * ncols + c0, nv, acc);
  }
}

template <int RPW, bool ALIGNED, int MODE>
__global__ void __launch_bounds__(256, MODE == 2 ? 3 : 4) k_spmm_bf16(
    const __nv_bfloat16* __restrict__ Xb, int64_t ldx, const float* __restrict__ X32,
    float* __restrict__ Y, int64_t nrows, int64_t ncols, const int64_t* __restrict__ rp,
    const int2* __restrict__ rec, const int64_t* __restrict__ srp, const int2* __restrict__ sl,
    const float* __restrict__ VT, const double* __restrict__ hd_row,
    const double* __restrict__ hd_col, double e_nuc, const float* __restrict__ Vrow,
    const uint64_t* __restrict__ scol, int n, int accumulate) {
  spmm_bf16_block<RPW, ALIGNED, MODE>(Xb, ldx, X32, Y, nrows, ncols, rp, rec, srp, sl, VT, hd_row,
                                      hd_col, e_nuc, Vrow, scol, n, accumulate, blockIdx.x,
                                      blockIdx.y);
}

// The same row product for several problems in one launch: problem r's blocks are
// [first[r], first[r+1]) of the flattened grid, cols_blocks[r] column tiles per row block.
struct SpmmJob {
  const float* X;
  float* Y;
  int64_t nrows, ncols;
  const int64_t* rp;
  const int2* rec;
  const int64_t* srp;
  const int2* sl;
  const float* VT;
  const double* hd_row;
  const double* hd_col;
  double e_nuc;
  const float* Vrow;
  const uint64_t* scol;
  int n, accumulate;
  int64_t col_blocks;
};

__device__ __forceinline__ int find_job(const int64_t* __restrict__ first, int R, int64_t b) {
  int lo = 0, hi = R;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (first[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

constexpr int kBatchRpw = 4;

// The jobs of one batched launch, passed by value as a kernel parameter (no host to
// device copy): kMaxJobs per launch, a longer batch is split.
constexpr int kMaxJobs = 48;
template <typename J>
struct JobTab {
  J job[kMaxJobs];
  int64_t first[kMaxJobs + 1];
  int R;
};

__global__ void __launch_bounds__(256, 4) k_spmm_rec4_batch(const __grid_constant__ JobTab<SpmmJob> tab) {
  const int64_t b = blockIdx.x;
  const int r = find_job(tab.first, tab.R, b);
  const SpmmJob& J = tab.job[r];
  const int64_t local = b - tab.first[r];
  if (J.ncols % 4 == 0)
    spmm_rec4_block<kBatchRpw, true>(J.X, J.Y, J.nrows, J.ncols, J.rp, J.rec, J.srp, J.sl, J.VT,
                                     J.hd_row, J.hd_col, J.e_nuc, J.Vrow, J.scol, J.n, J.accumulate,
                                     local % J.col_blocks, local / J.col_blocks);
  else
    spmm_rec4_block<kBatchRpw, false>(J.X, J.Y, J.nrows, J.ncols, J.rp, J.rec, J.srp, J.sl, J.VT,
                                      J.hd_row, J.hd_col, J.e_nuc, J.Vrow, J.scol, J.n, J.accumulate,
                                      local % J.col_blocks, local / J.col_blocks);
}

template <typename T>
const typename Rec<T>::type* recof(const hinqs_links_s* L);
template <>
const int2* recof<float>(const hinqs_links_s* L) { return L->rec32; }
template <>
const int4* recof<double>(const hinqs_links_s* L) { return L->rec64; }

// out[j][i] = in[i][j] (+ out[j][i] if accumulate) for in of rows x cols; 32x32 tiles.
template <typename T>
__device__ __forceinline__ void transpose_tile(const T* __restrict__ in, T* __restrict__ out,
                                               int64_t rows, int64_t cols, int accumulate,
                                               int64_t tx, int64_t ty) {
  __shared__ T tile[32][33];
  const int64_t bx = tx * 32, by = ty * 32;
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

template <typename T>
__global__ void k_transpose_t(const T* __restrict__ in, T* __restrict__ out, int64_t rows,
                              int64_t cols, int accumulate) {
  transpose_tile<T>(in, out, rows, cols, accumulate, blockIdx.x, blockIdx.y);
}

struct TransJob {
  const float* in;
  float* out;
  int64_t rows, cols, col_tiles;
};

// transposes of several problems in one launch (problem r's tiles [first[r], first[r+1]))
__global__ void k_transpose_batch(const __grid_constant__ JobTab<TransJob> tab) {
  const int64_t b = blockIdx.x;
  const int r = find_job(tab.first, tab.R, b);
  const TransJob& J = tab.job[r];
  const int64_t local = b - tab.first[r];
  transpose_tile<float>(J.in, J.out, J.rows, J.cols, 0, local % J.col_tiles, local / J.col_tiles);
}

// The BF16C same-spin stages of several problems in one launch each (problem r's
// blocks [first[r], first[r+1]) of the flattened grid).
struct BfJob {
  const __nv_bfloat16* Xb;
  int64_t ldx;
  const float* X32;
  float* Y;
  int64_t nrows, ncols;
  const int64_t* rp;
  const int2* rec;
  const int64_t* srp;
  const int2* sl;
  const float* VT;
  const double* hd_row;
  const double* hd_col;
  double e_nuc;
  const float* Vrow;
  const uint64_t* scol;
  int n, accumulate;
  int64_t col_blocks;
};

constexpr int kBfBatchRpw = 2;

template <int MODE>
__global__ void __launch_bounds__(256, MODE == 2 ? 3 : 4) k_spmm_bf16_batch(
    const __grid_constant__ JobTab<BfJob> tab) {
  const int64_t b = blockIdx.x;
  const int r = find_job(tab.first, tab.R, b);
  const BfJob& J = tab.job[r];
  const int64_t local = b - tab.first[r];
  if (J.ncols % 4 == 0)
    spmm_bf16_block<kBfBatchRpw, true, MODE>(J.Xb, J.ldx, J.X32, J.Y, J.nrows, J.ncols, J.rp,
                                             J.rec, J.srp, J.sl, J.VT, J.hd_row, J.hd_col, J.e_nuc,
                                             J.Vrow, J.scol, J.n, J.accumulate,
                                             local % J.col_blocks, local / J.col_blocks);
  else
    spmm_bf16_block<kBfBatchRpw, false, MODE>(J.Xb, J.ldx, J.X32, J.Y, J.nrows, J.ncols, J.rp,
                                              J.rec, J.srp, J.sl, J.VT, J.hd_row, J.hd_col,
                                              J.e_nuc, J.Vrow, J.scol, J.n, J.accumulate,
                                              local % J.col_blocks, local / J.col_blocks);
}

struct PackJob {
  const float* C;
  int64_t rows, cols;
  __nv_bfloat16* Cb;
  int64_t ldc;
  __nv_bfloat16* CTb;
  int64_t ldr;
  int64_t tiles_x;  // 32-column tiles over ldc
};

// k_bf16_pack over several problems (32 x 32 tiles covering ldc columns and ldr rows)
__global__ void k_bf16_pack_batch(const __grid_constant__ JobTab<PackJob> tab) {
  __shared__ float tile[32][33];
  const int64_t b = blockIdx.x;
  const int r = find_job(tab.first, tab.R, b);
  const PackJob& J = tab.job[r];
  const int64_t local = b - tab.first[r];
  const int64_t bx = (local % J.tiles_x) * 32, by = (local / J.tiles_x) * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = by + k, j = bx + threadIdx.x;
    const float v = (i < J.rows && j < J.cols) ? J.C[i * J.cols + j] : 0.f;
    tile[k][threadIdx.x] = v;
    if (i < J.rows && j < J.ldc) J.Cb[i * J.ldc + j] = __float2bfloat16_rn(v);
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t j = bx + k, i = by + threadIdx.x;
    if (j < J.cols && i < J.ldr) J.CTb[j * J.ldr + i] = __float2bfloat16_rn(tile[threadIdx.x][k]);
  }
}

struct AbArgs {
  int64_t Na, Nb;
  int n;
  const int64_t* a_srow;
  const int2* a_slink;
  const int2* b_ell;   // slot-major beta singles + self, [width][Nb]
  const int* b_cnt;    // entries per beta string
  int vec4;            // Nb % 4 == 0
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
    for (int64_t Ib0 = 0; Ib0 < A.Nb; Ib0 += blockDim.x) {
      const int64_t Ib = Ib0 + threadIdx.x;
      const bool live = Ib < A.Nb;
      T e[CH];
#pragma unroll
      for (int a = 0; a < CH; ++a) e[a] = T(0);
      const int nk = live ? A.b_cnt[Ib] : 0;
      const int2* ell = A.b_ell + Ib;
      int k = 0;
      for (; k + 2 <= nk; k += 2) {
        const int2 l0 = ell[(int64_t)k * A.Nb], l1 = ell[(int64_t)(k + 1) * A.Nb];
        T v0 = row[l0.x], v1 = row[l1.x];
        if (l0.y < 0) v0 = -v0;
        if (l1.y < 0) v1 = -v1;
        const T* er0 = eriT + ((l0.y > 0 ? l0.y : -l0.y) - 1) * LD;
        const T* er1 = eriT + ((l1.y > 0 ? l1.y : -l1.y) - 1) * LD;
        // two fused multiply-adds per column (not a product, a fma and an add)
#pragma unroll
        for (int a = 0; a < CH; ++a) e[a] = fma(v1, er1[a], fma(v0, er0[a], e[a]));
      }
      if (k < nk) {
        const int2 l0 = ell[(int64_t)k * A.Nb];
        T v0 = row[l0.x];
        if (l0.y < 0) v0 = -v0;
        const T* er0 = eriT + ((l0.y > 0 ? l0.y : -l0.y) - 1) * LD;
#pragma unroll
        for (int a = 0; a < CH; ++a) e[a] = fma(v0, er0[a], e[a]);
      }
      if constexpr (sizeof(T) == 4) {
        // transpose through shared memory, then float4 atomics over four
        // consecutive beta strings of one target row
        T* stage = Crow + (ROW_SMEM ? A.Nb : 0);  // [CH][256], 16-byte aligned
#pragma unroll
        for (int a = 0; a < CH; ++a) stage[a * 256 + threadIdx.x] = e[a];
        __syncthreads();
        for (int idx = threadIdx.x; idx < cnt * 64; idx += blockDim.x) {
          const int a = idx >> 6, m4 = (idx & 63) * 4;
          const int64_t ib = Ib0 + m4;
          if (ib >= A.Nb) continue;
          T* dst = sig + (int64_t)tgt[a] * A.Nb + ib;
          const T* src = stage + a * 256 + m4;
          if (A.vec4 && ib + 3 < A.Nb)
            atomicAdd(reinterpret_cast<float4*>(dst), make_float4(src[0], src[1], src[2], src[3]));
          else
            for (int q = 0; q < 4 && ib + q < A.Nb; ++q) atomicAdd(dst + q, src[q]);
        }
        __syncthreads();
      } else {
        if (live) {
#pragma unroll
          for (int a = 0; a < CH; ++a)
            if (a < cnt) atomicAdd(sig + (int64_t)tgt[a] * A.Nb + Ib, e[a]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// HINQS_PREC_FP64_DFAB: the opposite-spin term of an FP64 product in double-float
// arithmetic (df_fma and df_split in hinqs_internal.cuh): FP64 runs at 1/64 of the
// FP32 rate on this part, and a double-float multiply-add is about twelve FP32
// operations; the result carries about 1e-13 relative error, far below what the
// refinement residual of the mixed solver needs.

// The structure of k_sigma_ab (one block per alpha string Ja, CH alpha singles per
// pass, (pq|.) rows transposed in shared memory), with the rows and C split into
// double-float pairs once when they are staged and the sums kept as pairs.
template <int CH, bool ROW_SMEM>
__global__ void __launch_bounds__(256) k_sigma_ab_df(const double* __restrict__ C,
                                                     double* __restrict__ sig, AbArgs A,
                                                     const double* __restrict__ eri) {
  constexpr int LD = CH + 2;  // padded row of eriT (float2 entries)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n2 = A.n * A.n;
  float2* eriT = reinterpret_cast<float2*>(smem_raw);  // [n2][LD]
  int* tgt = reinterpret_cast<int*>(eriT + (size_t)n2 * LD);
  float2* Crow = reinterpret_cast<float2*>(tgt + CH + 4);  // [Nb]
  const int64_t Ja = blockIdx.x;
  const int64_t a_beg = A.a_srow[Ja], a_end = A.a_srow[Ja + 1];
  if (a_beg == a_end) return;
  const double* Cg = C + Ja * A.Nb;
  if (ROW_SMEM) {
    for (int64_t j = threadIdx.x; j < A.Nb; j += blockDim.x) Crow[j] = df_split(Cg[j]);
  }
  for (int64_t a0 = a_beg; a0 < a_end; a0 += CH) {
    const int cnt = (int)min64(CH, a_end - a0);
    __syncthreads();
    for (int i = threadIdx.x; i < n2 * CH; i += blockDim.x) {
      const int xy = i / CH, a = i % CH;
      double v = 0.0;
      if (a < cnt) {
        const int sp = A.a_slink[a0 + a].y;
        const int pq = (sp > 0 ? sp : -sp) - 1;
        v = eri[(int64_t)pq * n2 + xy];
        if (sp < 0) v = -v;
      }
      eriT[xy * LD + a] = df_split(v);
    }
    if (threadIdx.x < CH) tgt[threadIdx.x] = (threadIdx.x < cnt) ? A.a_slink[a0 + threadIdx.x].x : 0;
    __syncthreads();
    for (int64_t Ib0 = 0; Ib0 < A.Nb; Ib0 += blockDim.x) {
      const int64_t Ib = Ib0 + threadIdx.x;
      const bool live = Ib < A.Nb;
      float eh[CH], el[CH];
#pragma unroll
      for (int a = 0; a < CH; ++a) eh[a] = 0.f, el[a] = 0.f;
      const int nk = live ? A.b_cnt[Ib] : 0;
      const int2* ell = A.b_ell + Ib;
      for (int k = 0; k < nk; ++k) {
        const int2 l0 = ell[(int64_t)k * A.Nb];
        float2 v = ROW_SMEM ? Crow[l0.x] : df_split(Cg[l0.x]);
        if (l0.y < 0) v.x = -v.x, v.y = -v.y;
        const float2* er = eriT + ((l0.y > 0 ? l0.y : -l0.y) - 1) * LD;
#pragma unroll
        for (int a = 0; a < CH; ++a) {
          const float2 b = er[a];
          df_fma(v.x, v.y, b.x, b.y, eh[a], el[a]);
        }
      }
      if (live) {
#pragma unroll
        for (int a = 0; a < CH; ++a)
          if (a < cnt) atomicAdd(sig + (int64_t)tgt[a] * A.Nb + Ib, (double)eh[a] + (double)el[a]);
      }
    }
  }
}

// C (rows x cols, FP64) -> the double-float pair (hi, lo) of C and of its transpose,
// as separate FP32 arrays; 32 x 32 tiles.
__global__ void k_df_split_pack(const double* __restrict__ C, int64_t rows, int64_t cols,
                                float* __restrict__ hi, float* __restrict__ lo,
                                float* __restrict__ hiT, float* __restrict__ loT) {
  __shared__ double tile[32][33];
  const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = by + k, j = bx + threadIdx.x;
    if (i < rows && j < cols) {
      const double v = C[i * cols + j];
      tile[k][threadIdx.x] = v;
      const float2 d = df_split(v);
      hi[i * cols + j] = d.x;
      lo[i * cols + j] = d.y;
    }
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t j = bx + k, i = by + threadIdx.x;
    if (i < rows && j < cols) {
      const float2 d = df_split(tile[threadIdx.x][k]);
      hiT[j * rows + i] = d.x;
      loT[j * rows + i] = d.y;
    }
  }
}

// The same-spin row product of the FP64 mode in double-float arithmetic: four columns
// per lane (one 16-byte load of the high and one of the low parts per link), the FP64
// link records read 32 at a time and split into a pair once, by the lane that loaded
// them, before the warp shares them.  MODE 2 adds the diagonal term in FP64 (on the
// FP64 C), MODE 1 the alpha-self x beta-single term (VT as a pair, VT32 + VTlo32).
// Requires ncols % 4 == 0.
template <int RPW, int MODE>
__global__ void __launch_bounds__(256) k_spmm_df(
    const float* __restrict__ Xh, const float* __restrict__ Xl, const double* __restrict__ X64,
    double* __restrict__ Y, int64_t nrows, int64_t ncols, const int64_t* __restrict__ rp,
    const int4* __restrict__ rec, const int64_t* __restrict__ srp, const int2* __restrict__ sl,
    const float* __restrict__ VTh, const float* __restrict__ VTl,
    const double* __restrict__ hd_row, const double* __restrict__ hd_col, double e_nuc,
    const double* __restrict__ Vrow, const uint64_t* __restrict__ scol, int n, int accumulate) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = ((int64_t)blockIdx.x * 32 + lane) * 4;
  const bool active = c0 < ncols;
  const int64_t cc = active ? c0 : 0;
  const int n2 = n * n;
  const unsigned full = 0xffffffffu;
  const int64_t I0 = ((int64_t)blockIdx.y * kRowWarps + warp) * RPW;
  for (int rr = 0; rr < RPW; ++rr) {
    const int64_t I = I0 + rr;
    if (I >= nrows) break;  // warp-uniform
    float ah[4] = {0.f, 0.f, 0.f, 0.f}, al[4] = {0.f, 0.f, 0.f, 0.f};
    const int4* __restrict__ r = rec + rp[I];
    const int nk = (int)(rp[I + 1] - rp[I]);
    for (int k0 = 0; k0 < nk; k0 += 32) {
      int off = 0;
      float hh = 0.f, hl = 0.f;
      if (k0 + lane < nk) {
        const int4 q = __ldg(r + k0 + lane);
        off = q.x;
        const float2 d = df_split(__hiloint2double(q.w, q.z));
        hh = d.x, hl = d.y;
      }
      const int cnt = min(32, nk - k0);
      for (int u = 0; u < cnt; u += 4) {
        float4 xh[4], xl[4];
        float bh[4], bl[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int src = min(u + v, cnt - 1);
          const uint32_t o = (uint32_t)__shfl_sync(full, off, src);
          bh[v] = __shfl_sync(full, hh, src);
          bl[v] = __shfl_sync(full, hl, src);
          if (u + v >= cnt) bh[v] = 0.f, bl[v] = 0.f;
          xh[v] = __ldg(reinterpret_cast<const float4*>(Xh + o + cc));
          xl[v] = __ldg(reinterpret_cast<const float4*>(Xl + o + cc));
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          df_fma(bh[v], bl[v], xh[v].x, xl[v].x, ah[0], al[0]);
          df_fma(bh[v], bl[v], xh[v].y, xl[v].y, ah[1], al[1]);
          df_fma(bh[v], bl[v], xh[v].z, xl[v].z, ah[2], al[2]);
          df_fma(bh[v], bl[v], xh[v].w, xl[v].w, ah[3], al[3]);
        }
      }
    }
    if (MODE == 1 && active) {
      for (int64_t q = srp[I], qe = srp[I + 1]; q < qe; ++q) {
        const int2 l = sl[q];
        const int pair = (l.y > 0 ? l.y : -l.y) - 1;
        const float4 vh = __ldg(reinterpret_cast<const float4*>(VTh + (int64_t)pair * ncols + c0));
        const float4 vl = __ldg(reinterpret_cast<const float4*>(VTl + (int64_t)pair * ncols + c0));
        const float4 xh = __ldg(reinterpret_cast<const float4*>(Xh + (int64_t)l.x * ncols + c0));
        const float4 xl = __ldg(reinterpret_cast<const float4*>(Xl + (int64_t)l.x * ncols + c0));
        const float sg = l.y > 0 ? 1.f : -1.f;
        df_fma(sg * vh.x, sg * vl.x, xh.x, xl.x, ah[0], al[0]);
        df_fma(sg * vh.y, sg * vl.y, xh.y, xl.y, ah[1], al[1]);
        df_fma(sg * vh.z, sg * vl.z, xh.z, xl.z, ah[2], al[2]);
        df_fma(sg * vh.w, sg * vl.w, xh.w, xl.w, ah[3], al[3]);
      }
    }
    double y[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) y[v] = (double)ah[v] + (double)al[v];
    if constexpr (MODE == 2) {
      const double v0 = (lane < n) ? Vrow[I * n2 + lane * n + lane] : 0.0;
      const double v1 = (lane + 32 < n) ? Vrow[I * n2 + (lane + 32) * n + lane + 32] : 0.0;
      uint64_t b[4];
      double xs[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = active ? scol[cc + v] : 0;
      for (int j = 0; j < n; ++j) {
        const double a = __shfl_sync(full, j < 32 ? v0 : v1, j & 31);
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if ((b[v] >> j) & 1ull) xs[v] += a;
      }
      if (active) {
        const double hr = hd_row[I] + e_nuc;
#pragma unroll
        for (int v = 0; v < 4; ++v) y[v] = fma(hr + hd_col[c0 + v] + xs[v], X64[I * ncols + c0 + v], y[v]);
      }
    }
    if (active) {
      double* yo = Y + I * ncols + c0;
#pragma unroll
      for (int v = 0; v < 4; ++v) yo[v] = accumulate ? yo[v] + y[v] : y[v];
    }
  }
}

// The same-spin half of an FP64 product in double-float: false when it does not apply
// (records missing or a row length not a multiple of 4), and the caller takes FP64.
static bool spmm_df_fits(const hinqs_subspace_s* B, const hinqs_links_s* la,
                         const hinqs_links_s* lb) {
  return la->rec64 && lb->rec64 && la->VTlo32 && B->Na % 4 == 0 && B->Nb % 4 == 0;
}

static int spmm_df(const float* Xh, const float* Xl, const double* X64, double* Y, int64_t nrows,
                   int64_t ncols, const hinqs_links_s* L, const hinqs_links_s* Lsingles,
                   const float* VTh, const float* VTl, const double* hd_row, const double* hd_col,
                   double e_nuc, const double* Vrow, const uint64_t* scol, int n, int accumulate,
                   cudaStream_t s) {
  const int64_t* srp = Lsingles ? Lsingles->srow_ptr : nullptr;
  const int2* sl = Lsingles ? Lsingles->slink : nullptr;
  const int rpw = 2;
  const dim3 g((unsigned)ceil_div(ncols, 128), (unsigned)ceil_div(nrows, kRowWarps * rpw));
  auto go = [&](auto kern) {
    kern<<<g, 32 * kRowWarps, 0, s>>>(Xh, Xl, X64, Y, nrows, ncols, L->row_ptr, L->rec64, srp, sl,
                                      VTh, VTl, hd_row, hd_col, e_nuc, Vrow, scol, n, accumulate);
  };
  if (hd_row) go(k_spmm_df<2, 2>);
  else if (srp) go(k_spmm_df<2, 1>);
  else go(k_spmm_df<2, 0>);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

template <int CH>
static int launch_ab_df(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                        const hinqs_links_s* lb, const double* c, double* sig, cudaStream_t s,
                        size_t smem_limit) {
  AbArgs A{B->Na, B->Nb, H->n, la->srow_ptr, la->slink, lb->sell, lb->scount, B->Nb % 4 == 0};
  const int n2 = H->n * H->n;
  size_t base = (size_t)n2 * (CH + 2) * sizeof(float2) + (CH + 4) * sizeof(int);
  base = (base + 15) & ~(size_t)15;
  const size_t with_row = base + (((size_t)B->Nb * sizeof(float2) + 15) & ~(size_t)15);
  if (with_row <= smem_limit) {
    auto kern = k_sigma_ab_df<CH, true>;
    HQ_TRY(allow_max_smem(kern));
    kern<<<(unsigned)B->Na, 256, with_row, s>>>(c, sig, A, H->eri);
  } else {
    auto kern = k_sigma_ab_df<CH, false>;
    HQ_TRY(allow_max_smem(kern));
    kern<<<(unsigned)B->Na, 256, base, s>>>(c, sig, A, H->eri);
  }
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

template <typename T, int CH>
static int launch_ab(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                     const hinqs_links_s* lb, const T* c, T* sig, cudaStream_t s,
                     size_t smem_limit) {
  AbArgs A{B->Na, B->Nb, H->n, la->srow_ptr, la->slink, lb->sell, lb->scount, B->Nb % 4 == 0};
  const int n2 = H->n * H->n;
  constexpr int LD = CH + 16 / (int)sizeof(T);
  size_t base = (size_t)n2 * LD * sizeof(T) + (CH + 4) * sizeof(int);
  base = (base + 15) & ~(size_t)15;
  if (sizeof(T) == 4) base += (size_t)CH * 256 * sizeof(T);  // epilogue staging
  size_t with_row = base + (((size_t)B->Nb * sizeof(T) + 15) & ~(size_t)15);
  if (with_row <= smem_limit) {
    auto kern = k_sigma_ab<T, CH, true>;
    HQ_TRY(allow_max_smem(kern));
    kern<<<(unsigned)B->Na, 256, with_row, s>>>(c, sig, A, Prec<T>::eri(H));
  } else {
    auto kern = k_sigma_ab<T, CH, false>;
    HQ_TRY(allow_max_smem(kern));
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
  const auto* rec = recof<T>(L);
  if constexpr (sizeof(T) == 4) {
    if (rec && ncols % 4 == 0) {
      const int64_t* srp = Lsingles ? Lsingles->srow_ptr : nullptr;
      const int2* sl = Lsingles ? Lsingles->slink : nullptr;
      const int rpw = L->tune_rows ? L->tune_rows : kRowsPerWarp;
      auto go = [&](auto kern, int r) {
        const dim3 g((unsigned)ceil_div(ncols, 128), (unsigned)ceil_div(nrows, kRowWarps * r));
        kern<<<g, 32 * kRowWarps, 0, s>>>(X, Y, nrows, ncols, L->row_ptr, rec, srp, sl, VT, hd_row,
                                          hd_col, e_nuc, Vrow, scol, n, accumulate);
      };
      if (rpw == 2) go(k_spmm_rec4<2>, 2);
      else if (rpw == 8) go(k_spmm_rec4<8>, 8);
      else go(k_spmm_rec4<4>, 4);
      HQ_LAUNCH_CHECK();
      return HINQS_OK;
    }
  }
  if (rec) {
    const int64_t* srp = Lsingles ? Lsingles->srow_ptr : nullptr;
    const int2* sl = Lsingles ? Lsingles->slink : nullptr;
    const int rpw = L->tune_rows ? L->tune_rows : kRowsPerWarp;
    auto go = [&](auto kern, int vec, int r) {
      const unsigned gy = (unsigned)ceil_div(nrows, kRowWarps * r);
      kern<<<dim3((unsigned)ceil_div(ncols, 32 * vec), gy), 32 * kRowWarps, 0, s>>>(
          X, Y, nrows, ncols, L->row_ptr, rec, srp, sl, VT, hd_row, hd_col, e_nuc, Vrow, scol, n,
          accumulate);
    };
    if (ncols % 2 == 0) {
      if (rpw == 2) go(k_spmm_rec<T, 2, 2>, 2, 2);
      else if (rpw == 8) go(k_spmm_rec<T, 2, 8>, 2, 8);
      else go(k_spmm_rec<T, 2, 4>, 2, 4);
    } else {
      if (rpw == 2) go(k_spmm_rec<T, 1, 2>, 1, 2);
      else if (rpw == 8) go(k_spmm_rec<T, 1, 8>, 1, 8);
      else go(k_spmm_rec<T, 1, 4>, 1, 4);
    }
    HQ_LAUNCH_CHECK();
    return HINQS_OK;
  }
  dim3 grid((unsigned)ceil_div(ncols, 32), (unsigned)ceil_div(nrows, kRowWarps * kRowsPerWarp));
  k_spmm_rows<T><<<grid, 32 * kRowWarps, 0, s>>>(
      X, Y, nrows, ncols, L->row_ptr, L->col, Prec<T>::hval(L),
      Lsingles ? Lsingles->srow_ptr : nullptr, Lsingles ? Lsingles->slink : nullptr, VT, hd_row,
      hd_col, e_nuc, Vrow, scol, n, accumulate);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

constexpr int kDoubleFloat = -1;  // sigma_impl<double>: opposite-spin term in double-float

template <typename T>
static int sigma_impl(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                      const hinqs_links_s* lb, const T* c, T* sig, cudaStream_t s,
                      int tc_split, int parts) {
  const size_t limit = 200 * 1024;
  const int n = H->n, n2 = n * n;
  const int64_t Na = B->Na, Nb = B->Nb, N = Na * Nb;
  T *CT = nullptr, *ST = nullptr, *DFT = nullptr;
  int rc = HINQS_OK;
  // double-float same-spin half: CT holds the (hi, lo) pair of C, DFT that of C^T
  bool df_same = false;
  if constexpr (sizeof(T) == 8) df_same = tc_split == kDoubleFloat && spmm_df_fits(B, la, lb);
  if ((parts & kSameSpin) && ((rc = dalloc(&CT, N, s)) || (rc = dalloc(&ST, N, s)) ||
                              (df_same && (rc = dalloc(&DFT, N, s))))) {
    dfree(CT, s);
    dfree(ST, s);
    dfree(DFT, s);
    return rc;
  }
  auto run = [&]() -> int {
    if (!(parts & kSameSpin)) goto opposite;
    if constexpr (sizeof(T) == 8) {
      if (df_same) {
        float* Xh = reinterpret_cast<float*>(CT);
        float* XhT = reinterpret_cast<float*>(DFT);
        const dim3 tg((unsigned)ceil_div(Nb, 32), (unsigned)ceil_div(Na, 32));
        k_df_split_pack<<<tg, dim3(32, 8), 0, s>>>(c, Na, Nb, Xh, Xh + N, XhT, XhT + N);
        HQ_LAUNCH_CHECK();
        // beta same-spin links and alpha-self x beta singles, rows = beta strings
        HQ_TRY(spmm_df(XhT, XhT + N, nullptr, ST, Nb, Na, lb, lb, la->VT32, la->VTlo32, nullptr,
                       nullptr, 0.0, nullptr, nullptr, n, 0, s));
        HQ_TRY(transpose<T>(ST, sig, Nb, Na, 0, s));
        // alpha same-spin links and the diagonal, rows = alpha strings
        HQ_TRY(spmm_df(Xh, Xh + N, c, sig, Na, Nb, la, nullptr, nullptr, nullptr, la->hdiag,
                       lb->hdiag, H->e_nuc, la->V64, B->sb, n, 1, s));
        goto opposite;
      }
    }
    HQ_TRY(transpose<T>(c, CT, Na, Nb, 0, s));
    // beta same-spin links and alpha-self x beta singles, rows = beta strings
    HQ_TRY(spmm_rows<T>(CT, ST, Nb, Na, lb, lb, VTof<T>(la), nullptr, nullptr, 0.0, nullptr,
                        nullptr, n, 0, s));
    HQ_TRY(transpose<T>(ST, sig, Nb, Na, 0, s));
    // alpha same-spin links and the diagonal, rows = alpha strings
    HQ_TRY(spmm_rows<T>(c, sig, Na, Nb, la, nullptr, nullptr, la->hdiag, lb->hdiag, H->e_nuc,
                        Prec<T>::V(la), B->sb, n, 1, s));
  opposite:
    if (!(parts & kOppositeSpin) || la->nsingle == 0) return HINQS_OK;
    if constexpr (sizeof(T) == 4) {
      if (tc_split) {
        const int r = sigma_ab_tc_launch(H, B, la, lb, c, sig, tc_split, s);
        if (r != kTcNoFit) return r;
      }
    } else {
      if (tc_split == kDoubleFloat) {  // the opposite-spin term in double-float
        const int ch = (size_t)n2 * 18 * sizeof(float2) + 256 <= limit / 2 ? 16 : 8;
        return ch == 16 ? launch_ab_df<16>(H, B, la, lb, c, sig, s, limit)
                        : launch_ab_df<8>(H, B, la, lb, c, sig, s, limit);
      }
    }
    auto need = [&](int ch) { return (size_t)n2 * (ch + 16 / sizeof(T)) * sizeof(T) + 256; };
    int ch = la->tune_ch ? la->tune_ch : (sizeof(T) == 4 ? 32 : 16);
    if (ch == 32 && !(need(32) <= limit / 2)) ch = 16;
    if (ch == 16 && !(need(16) <= limit / 2)) ch = 8;
    if (ch == 32) return launch_ab<T, 32>(H, B, la, lb, c, sig, s, limit);
    if (ch == 16) return launch_ab<T, 16>(H, B, la, lb, c, sig, s, limit);
    return launch_ab<T, 8>(H, B, la, lb, c, sig, s, limit);
  };
  rc = run();
  dfree(CT, s);
  dfree(ST, s);
  dfree(DFT, s);
  return rc;
}

// One row product on the BF16 operand (rows per warp from the links' tuning).
static int spmm_bf16(const __nv_bfloat16* Xb, int64_t ldx, const float* X32, float* Y,
                     int64_t nrows, int64_t ncols, const hinqs_links_s* L,
                     const hinqs_links_s* Lsingles, const float* VT, const double* hd_row,
                     const double* hd_col, double e_nuc, const float* Vrow, const uint64_t* scol,
                     int n, int accumulate, cudaStream_t s) {
  const int64_t* srp = Lsingles ? Lsingles->srow_ptr : nullptr;
  const int2* sl = Lsingles ? Lsingles->slink : nullptr;
  const int rpw = L->tune_rows ? L->tune_rows : kRowsPerWarp;
  auto go = [&](auto kern, int r) {
    const dim3 g((unsigned)ceil_div(ncols, 256), (unsigned)ceil_div(nrows, kRowWarps * r));
    kern<<<g, 32 * kRowWarps, 0, s>>>(Xb, ldx, X32, Y, nrows, ncols, L->row_ptr, L->rec16, srp,
                                      sl, VT, hd_row, hd_col, e_nuc, Vrow, scol, n, accumulate);
  };
  auto by_rows = [&](auto k2, auto k4, auto k8) {
    if (rpw == 2) go(k2, 2);
    else if (rpw == 8) go(k8, 8);
    else go(k4, 4);
  };
  const int mode = hd_row ? 2 : (srp ? 1 : 0);
  if (ncols % 4 == 0) {
    if (mode == 2) by_rows(k_spmm_bf16<2, true, 2>, k_spmm_bf16<4, true, 2>, k_spmm_bf16<8, true, 2>);
    else if (mode == 1) by_rows(k_spmm_bf16<2, true, 1>, k_spmm_bf16<4, true, 1>, k_spmm_bf16<8, true, 1>);
    else by_rows(k_spmm_bf16<2, true, 0>, k_spmm_bf16<4, true, 0>, k_spmm_bf16<8, true, 0>);
  } else {
    if (mode == 2) by_rows(k_spmm_bf16<2, false, 2>, k_spmm_bf16<4, false, 2>, k_spmm_bf16<8, false, 2>);
    else if (mode == 1) by_rows(k_spmm_bf16<2, false, 1>, k_spmm_bf16<4, false, 1>, k_spmm_bf16<8, false, 1>);
    else by_rows(k_spmm_bf16<2, false, 0>, k_spmm_bf16<4, false, 0>, k_spmm_bf16<8, false, 0>);
  }
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

// HINQS_PREC_FP32_BF16C: the same-spin half on BF16 copies of C and C^T (rows padded
// to 64 elements), the opposite-spin half as HINQS_PREC_FP32_BF16AB.  Links without
// BF16 records (N * padded row >= 2^32) take the FP32 same-spin half instead.
static int sigma_bf16c(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                       const hinqs_links_s* lb, const float* c, float* sig, cudaStream_t s,
                       int parts) {
  if (!la->rec16 || !lb->rec16 || !la->rec32 || !lb->rec32) {
    HQ_TRY(sigma_impl<float>(H, B, la, lb, c, sig, s, 1, parts & kSameSpin));
    return (parts & kOppositeSpin) ? sigma_impl<float>(H, B, la, lb, c, sig, s, 1, kOppositeSpin)
                                   : HINQS_OK;
  }
  if (parts & kSameSpin) {
    const int64_t Na = B->Na, Nb = B->Nb, ldc = la->ld16, ldr = lb->ld16;
    __nv_bfloat16 *Cb = nullptr, *CTb = nullptr;
    float* ST = nullptr;
    int rc = HINQS_OK;
    if (!(rc = dalloc(&Cb, (size_t)(Na * ldc), s)) && !(rc = dalloc(&CTb, (size_t)(Nb * ldr), s)) &&
        !(rc = dalloc(&ST, (size_t)(Na * Nb), s))) {
      auto run = [&]() -> int {
        const dim3 tg((unsigned)ceil_div(ldc, 32), (unsigned)ceil_div(ldr, 32));
        k_bf16_pack<<<tg, dim3(32, 8), 0, s>>>(c, Na, Nb, Cb, ldc, CTb, ldr);
        HQ_LAUNCH_CHECK();
        // beta same-spin links and alpha-self x beta singles, rows = beta strings
        HQ_TRY(spmm_bf16(CTb, ldr, nullptr, ST, Nb, Na, lb, lb, la->VT32, nullptr, nullptr, 0.0,
                         nullptr, nullptr, H->n, 0, s));
        HQ_TRY(transpose<float>(ST, sig, Nb, Na, 0, s));
        // alpha same-spin links and the diagonal, rows = alpha strings
        return spmm_bf16(Cb, ldc, c, sig, Na, Nb, la, nullptr, nullptr, la->hdiag, lb->hdiag,
                         H->e_nuc, la->V32, B->sb, H->n, 1, s);
      };
      rc = run();
    }
    dfree(Cb, s);
    dfree(CTb, s);
    dfree(ST, s);
    HQ_TRY(rc);
  }
  return (parts & kOppositeSpin) ? sigma_impl<float>(H, B, la, lb, c, sig, s, 1, kOppositeSpin)
                                 : HINQS_OK;
}

// Launch the jobs in tables of kMaxJobs; per_job(i, job) fills job i and returns its
// block count.
template <typename J, typename Fill, typename Kern>
static int launch_jobs(int R, Fill per_job, Kern kern, dim3 block, cudaStream_t s) {
  for (int r0 = 0; r0 < R; r0 += kMaxJobs) {
    JobTab<J> tab;
    tab.R = std::min(kMaxJobs, R - r0);
    tab.first[0] = 0;
    for (int i = 0; i < tab.R; ++i) tab.first[i + 1] = tab.first[i] + per_job(r0 + i, tab.job[i]);
    if (tab.first[tab.R] == 0) continue;
    kern<<<(unsigned)tab.first[tab.R], block, 0, s>>>(tab);
    HQ_LAUNCH_CHECK();
  }
  return HINQS_OK;
}

int sigma_batch_launch(const SigmaReq* reqs, int n, cudaStream_t s) {
  // f32: same-spin half in FP32 row products (FP32, BF16AB, BF16X3AB); bfc: on BF16
  // copies of C (BF16C); the rest one problem at a time
  std::vector<int> f32, bfc;
  for (int i = 0; i < n; ++i) {
    const SigmaReq& r = reqs[i];
    const bool solo = r.precision == HINQS_PREC_FP64 || r.precision == HINQS_PREC_FP64_DFAB ||
                      !r.la->rec32 || !r.lb->rec32 || r.B->Na * r.B->Nb >= kBatchSoloN ||
                      (r.precision == HINQS_PREC_FP32_BF16C && (!r.la->rec16 || !r.lb->rec16));
    if (solo) HQ_TRY(sigma_launch(r.H, r.B, r.la, r.lb, r.x, r.y, r.precision, s));
    else if (r.precision == HINQS_PREC_FP32_BF16C) bfc.push_back(i);
    else f32.push_back(i);
  }
  if (f32.empty() && bfc.empty()) return HINQS_OK;
  const int R = (int)f32.size(), RB = (int)bfc.size();
  std::vector<float*> CT(R, nullptr), ST(R, nullptr), STb(RB, nullptr);
  std::vector<__nv_bfloat16*> Cb(RB, nullptr), CTb(RB, nullptr);
  auto run = [&]() -> int {
    for (int i = 0; i < R; ++i) {
      const int64_t N = reqs[f32[i]].B->Na * reqs[f32[i]].B->Nb;
      HQ_TRY(dalloc(&CT[i], N, s));
      HQ_TRY(dalloc(&ST[i], N, s));
    }
    for (int i = 0; i < RB; ++i) {
      const SigmaReq& r = reqs[bfc[i]];
      HQ_TRY(dalloc(&Cb[i], (size_t)(r.B->Na * r.la->ld16), s));
      HQ_TRY(dalloc(&CTb[i], (size_t)(r.B->Nb * r.lb->ld16), s));
      HQ_TRY(dalloc(&STb[i], (size_t)(r.B->Na * r.B->Nb), s));
    }
    // a transpose stage over requests: in (rows x cols) -> out
    auto transpose_all = [&](const std::vector<int>& ids, bool forward,
                             const std::vector<float*>& tmp_in,
                             const std::vector<float*>& tmp_out) -> int {
      auto fill = [&](int i, TransJob& j) -> int64_t {
        const SigmaReq& r = reqs[ids[i]];
        const int64_t rows = forward ? r.B->Na : r.B->Nb, cols = forward ? r.B->Nb : r.B->Na;
        j = TransJob{forward ? static_cast<const float*>(r.x) : tmp_in[i],
                     forward ? tmp_out[i] : static_cast<float*>(r.y), rows, cols,
                     ceil_div(cols, 32)};
        return j.col_tiles * ceil_div(rows, 32);
      };
      return launch_jobs<TransJob>((int)ids.size(), fill, k_transpose_batch, dim3(32, 8), s);
    };
    // a row-product stage over every request: beta rows on C^T, or alpha rows on C
    auto rows_all = [&](bool beta) -> int {
      auto fill = [&](int i, SpmmJob& j) -> int64_t {
        const SigmaReq& r = reqs[f32[i]];
        const hinqs_links_s* L = beta ? r.lb : r.la;
        j = SpmmJob{};
        j.X = beta ? CT[i] : static_cast<const float*>(r.x);
        j.Y = beta ? ST[i] : static_cast<float*>(r.y);
        j.nrows = beta ? r.B->Nb : r.B->Na;
        j.ncols = beta ? r.B->Na : r.B->Nb;
        j.rp = L->row_ptr;
        j.rec = L->rec32;
        j.srp = beta ? r.lb->srow_ptr : nullptr;
        j.sl = beta ? r.lb->slink : nullptr;
        j.VT = beta ? r.la->VT32 : nullptr;
        j.hd_row = beta ? nullptr : r.la->hdiag;
        j.hd_col = beta ? nullptr : r.lb->hdiag;
        j.e_nuc = beta ? 0.0 : r.H->e_nuc;
        j.Vrow = beta ? nullptr : r.la->V32;
        j.scol = beta ? nullptr : r.B->sb;
        j.n = r.H->n;
        j.accumulate = beta ? 0 : 1;
        j.col_blocks = ceil_div(j.ncols, 128);
        return j.col_blocks * ceil_div(j.nrows, kRowWarps * kBatchRpw);
      };
      return launch_jobs<SpmmJob>(R, fill, k_spmm_rec4_batch, dim3(32 * kRowWarps), s);
    };
    if (R > 0) {
      HQ_TRY(transpose_all(f32, true, CT, CT));    // C^T
      HQ_TRY(rows_all(true));                      // beta same-spin + alpha self x beta singles
      HQ_TRY(transpose_all(f32, false, ST, ST));   // sigma = (...)^T
      HQ_TRY(rows_all(false));                     // += alpha same-spin + diagonal
    }
    if (RB > 0) {
      // BF16 copies of C and C^T, then the row products on them (as sigma_bf16c)
      auto pack = [&](int i, PackJob& j) -> int64_t {
        const SigmaReq& r = reqs[bfc[i]];
        j = PackJob{static_cast<const float*>(r.x), r.B->Na, r.B->Nb, Cb[i], r.la->ld16, CTb[i],
                    r.lb->ld16, ceil_div(r.la->ld16, 32)};
        return j.tiles_x * ceil_div(r.lb->ld16, 32);
      };
      HQ_TRY(launch_jobs<PackJob>(RB, pack, k_bf16_pack_batch, dim3(32, 8), s));
      auto bf_rows = [&](bool beta) -> int {
        auto fill = [&](int i, BfJob& j) -> int64_t {
          const SigmaReq& r = reqs[bfc[i]];
          const hinqs_links_s* L = beta ? r.lb : r.la;
          j = BfJob{};
          j.Xb = beta ? CTb[i] : Cb[i];
          j.ldx = beta ? r.lb->ld16 : r.la->ld16;
          j.X32 = beta ? nullptr : static_cast<const float*>(r.x);
          j.Y = beta ? STb[i] : static_cast<float*>(r.y);
          j.nrows = beta ? r.B->Nb : r.B->Na;
          j.ncols = beta ? r.B->Na : r.B->Nb;
          j.rp = L->row_ptr;
          j.rec = L->rec16;
          j.srp = beta ? r.lb->srow_ptr : nullptr;
          j.sl = beta ? r.lb->slink : nullptr;
          j.VT = beta ? r.la->VT32 : nullptr;
          j.hd_row = beta ? nullptr : r.la->hdiag;
          j.hd_col = beta ? nullptr : r.lb->hdiag;
          j.e_nuc = beta ? 0.0 : r.H->e_nuc;
          j.Vrow = beta ? nullptr : r.la->V32;
          j.scol = beta ? nullptr : r.B->sb;
          j.n = r.H->n;
          j.accumulate = beta ? 0 : 1;
          j.col_blocks = ceil_div(j.ncols, 256);
          return j.col_blocks * ceil_div(j.nrows, kRowWarps * kBfBatchRpw);
        };
        return beta ? launch_jobs<BfJob>(RB, fill, k_spmm_bf16_batch<1>, dim3(32 * kRowWarps), s)
                    : launch_jobs<BfJob>(RB, fill, k_spmm_bf16_batch<2>, dim3(32 * kRowWarps), s);
      };
      HQ_TRY(bf_rows(true));                          // beta rows on C^T -> STb
      HQ_TRY(transpose_all(bfc, false, STb, STb));    // sigma = STb^T
      HQ_TRY(bf_rows(false));                         // += alpha rows + diagonal
    }
    // the opposite-spin term: one tensor-core launch per split mode, the rest singly
    std::vector<int> all_fp32(f32);
    all_fp32.insert(all_fp32.end(), bfc.begin(), bfc.end());
    for (int split : {1, 3}) {
      std::vector<int> ids;
      for (int i : all_fp32) {
        const int p = reqs[i].precision;
        const bool take = split == 1 ? (p == HINQS_PREC_FP32_BF16AB || p == HINQS_PREC_FP32_BF16C)
                                     : p == HINQS_PREC_FP32_BF16X3AB;
        if (take && reqs[i].la->nsingle > 0) ids.push_back(i);
      }
      if (ids.empty()) continue;
      const int rc = sigma_ab_tc_batch(reqs, ids.data(), (int)ids.size(), split, s);
      if (rc < 0) return rc;
      if (rc == kTcNoFit)
        for (int i : ids)
          HQ_TRY(sigma_launch(reqs[i].H, reqs[i].B, reqs[i].la, reqs[i].lb, reqs[i].x, reqs[i].y,
                              reqs[i].precision, s, kOppositeSpin));
    }
    for (int i : f32)
      if (reqs[i].precision == HINQS_PREC_FP32 && reqs[i].la->nsingle > 0)
        HQ_TRY(sigma_launch(reqs[i].H, reqs[i].B, reqs[i].la, reqs[i].lb, reqs[i].x, reqs[i].y,
                            reqs[i].precision, s, kOppositeSpin));
    return HINQS_OK;
  };
  const int rc = run();
  for (int i = 0; i < R; ++i) {
    dfree(CT[i], s);
    dfree(ST[i], s);
  }
  for (int i = 0; i < RB; ++i) {
    dfree(Cb[i], s);
    dfree(CTb[i], s);
    dfree(STb[i], s);
  }
  return rc;
}

int sigma_launch(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                 const hinqs_links_s* lb, const void* c, void* sigma, int precision,
                 cudaStream_t s, int parts) {
  if (precision == HINQS_PREC_FP64)
    return sigma_impl<double>(H, B, la, lb, (const double*)c, (double*)sigma, s, 0, parts);
  if (precision == HINQS_PREC_FP64_DFAB)
    return sigma_impl<double>(H, B, la, lb, (const double*)c, (double*)sigma, s, kDoubleFloat,
                              parts);
  if (precision == HINQS_PREC_FP32)
    return sigma_impl<float>(H, B, la, lb, (const float*)c, (float*)sigma, s, 0, parts);
  if (precision == HINQS_PREC_FP32_BF16AB)
    return sigma_impl<float>(H, B, la, lb, (const float*)c, (float*)sigma, s, 1, parts);
  if (precision == HINQS_PREC_FP32_BF16X3AB)
    return sigma_impl<float>(H, B, la, lb, (const float*)c, (float*)sigma, s, 3, parts);
  if (precision == HINQS_PREC_FP32_BF16C)
    return sigma_bf16c(H, B, la, lb, (const float*)c, (float*)sigma, s, parts);
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

extern "C" int hinqs_sigma_workspace_size(int64_t n_alpha_strings, int64_t n_beta_strings,
                                          int precision, size_t* bytes) {
  if (!bytes || n_alpha_strings < 0 || n_beta_strings < 0)
    return fail(HINQS_ERR_ARG, "hinqs_sigma_workspace_size: NULL output or negative size");
  if (precision < HINQS_PREC_FP64 || precision > HINQS_PREC_FP64_DFAB)
    return fail(HINQS_ERR_ARG, "hinqs_sigma_workspace_size: unknown precision %d", precision);
  // the transposed vector and the transposed partial result of the same-spin half
  // (BF16C: the two padded BF16 copies and the transposed FP32 partial result)
  const size_t elem = (precision == HINQS_PREC_FP64 || precision == HINQS_PREC_FP64_DFAB)
                          ? sizeof(double) : sizeof(float);
  *bytes = 2 * (size_t)(n_alpha_strings * n_beta_strings) * elem;
  if (precision == HINQS_PREC_FP64_DFAB)  // plus the pair (hi, lo) of C^T
    *bytes = 3 * (size_t)(n_alpha_strings * n_beta_strings) * sizeof(double);
  if (precision == HINQS_PREC_FP32_BF16C) {
    const size_t pa = (size_t)(n_alpha_strings + 63) / 64 * 64;
    const size_t pb = (size_t)(n_beta_strings + 63) / 64 * 64;
    *bytes = 2 * ((size_t)n_alpha_strings * pb + (size_t)n_beta_strings * pa) +
             4 * (size_t)(n_alpha_strings * n_beta_strings);
  }
  return HINQS_OK;
}

static int sigma_entry(const hinqs_ham* H, const hinqs_subspace* B, const hinqs_links* la,
                       const hinqs_links* lb, const void* c, void* sigma, int precision,
                       void* stream, int parts, const char* who) {
  HQ_TRY(check_triplet(H, B, la, lb, who));
  if (!c || !sigma) return fail(HINQS_ERR_ARG, "%s: NULL vector", who);
  if (c == sigma) return fail(HINQS_ERR_ARG, "%s: c and sigma must not overlap", who);
  HQ_TRY(sigma_launch(H, B, la, lb, c, sigma, precision, (cudaStream_t)stream, parts));
  if ((parts & kOppositeSpin) &&
      (precision == HINQS_PREC_FP32_BF16AB || precision == HINQS_PREC_FP32_BF16X3AB ||
       precision == HINQS_PREC_FP32_BF16C))
    return tc_error_check((cudaStream_t)stream);
  return HINQS_OK;
}

extern "C" int hinqs_sigma_batch(int n, const hinqs_ham* const* hams,
                                 const hinqs_subspace* const* subs, const hinqs_links* const* las,
                                 const hinqs_links* const* lbs, const void* const* cs,
                                 void* const* sigmas, int precision, void* stream) {
  if (n < 0 || (n > 0 && (!hams || !subs || !las || !lbs || !cs || !sigmas)))
    return fail(HINQS_ERR_ARG, "hinqs_sigma_batch: NULL arrays");
  if (precision < HINQS_PREC_FP64 || precision > HINQS_PREC_FP64_DFAB)
    return fail(HINQS_ERR_ARG, "hinqs_sigma_batch: unknown precision %d", precision);
  std::vector<SigmaReq> reqs;
  for (int g = 0; g < n; ++g) {
    HQ_TRY(check_triplet(hams[g], subs[g], las[g], lbs[g], "hinqs_sigma_batch"));
    if (!cs[g] || !sigmas[g] || cs[g] == sigmas[g])
      return fail(HINQS_ERR_ARG, "hinqs_sigma_batch: problem %d: NULL or overlapping vectors", g);
    reqs.push_back(SigmaReq{hams[g], subs[g], las[g], lbs[g], cs[g], sigmas[g], precision});
  }
  if (n == 0) return HINQS_OK;
  HQ_TRY(sigma_batch_launch(reqs.data(), n, (cudaStream_t)stream));
  if (precision == HINQS_PREC_FP32_BF16AB || precision == HINQS_PREC_FP32_BF16X3AB ||
      precision == HINQS_PREC_FP32_BF16C)
    return tc_error_check((cudaStream_t)stream);
  return HINQS_OK;
}

extern "C" int hinqs_sigma(const hinqs_ham* H, const hinqs_subspace* B, const hinqs_links* la,
                           const hinqs_links* lb, const void* c, void* sigma, int precision,
                           void* stream) {
  return sigma_entry(H, B, la, lb, c, sigma, precision, stream, kSameSpin | kOppositeSpin,
                     "hinqs_sigma");
}

extern "C" int hinqs_sigma_same_spin(const hinqs_ham* H, const hinqs_subspace* B,
                                     const hinqs_links* la, const hinqs_links* lb, const void* c,
                                     void* sigma, int precision, void* stream) {
  return sigma_entry(H, B, la, lb, c, sigma, precision, stream, kSameSpin,
                     "hinqs_sigma_same_spin");
}

extern "C" int hinqs_sigma_opposite_spin(const hinqs_ham* H, const hinqs_subspace* B,
                                         const hinqs_links* la, const hinqs_links* lb,
                                         const void* c, void* sigma, int precision, void* stream) {
  return sigma_entry(H, B, la, lb, c, sigma, precision, stream, kOppositeSpin,
                     "hinqs_sigma_opposite_spin");
}
