// K8: Davidson eigensolver (Step 3) on the device, FP64 and mixed precision.
//
// FP64 mode: the textbook method.  Basis V (orthonormal, FP64), W = H V, projected
// matrix G = V^T W (FP64, m x m), lowest Ritz pair (theta, y) by parallel cyclic
// Jacobi in one thread block, residual r = W y - theta V y, correction
// t = r / (H_diag - theta) with |H_diag - theta| floored, classical Gram-Schmidt
// twice, restart at m_max keeping the current and previous Ritz vectors.
//
// Mixed mode (FP32 bulk, FP64 refinement): outer cycles keep an FP64 unit
// vector x with its FP64 product s = H x.  Each cycle solves for the correction in
// the subspace {x} + span{v_1..v_m}, where the v_i and w_i = H v_i are FP32
// (FP32 sigma) and the projected matrix is FP64 with G_00 = x.s, G_0i = s.v_i
// (exact coupling through the FP64 product and the symmetry of H) and
// G_ij = v_i.w_j.  The cycle's Ritz vector becomes the next x.  Rounding in the
// FP32 products enters only through the correction, so every cycle gains
// accuracy until the FP64 residual meets the tolerance.
#include <algorithm>
#include <chrono>
#include <type_traits>
#include <cmath>
#include <vector>

#include "hinqs_internal.cuh"

namespace hinqs {

int check_triplet(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                  const hinqs_links_s* lb, const char* who);

constexpr int kMaxSub = 32;
constexpr int kRRThreads = 128;  // threads of the projected eigensolver
constexpr int kRitzStride = kMaxSub + 2;  // (theta, y[kMaxSub], pad) per Ritz pair
constexpr int kRedGrid = 2 * kNumSMs;   // blocks per vector of the dot products
constexpr int kResGrid = 8 * kNumSMs;   // blocks of the residual pass (one vector pair)
constexpr int kRedThreads = 256;
constexpr int kDefaultKeepFp64 = 4;   // vectors kept at a restart (restart_keep = 0)
constexpr int kDefaultKeepMixed = 4;

// ---------------------------------------------------------------- kernels --

// The block that finishes last among the gridDim.x blocks of one output sums that
// output's partials in a fixed order (lane-strided, then a shuffle tree, so the
// result does not depend on which block came last) and re-arms the counter.
__device__ __forceinline__ void last_block_reduce(const double* __restrict__ partial, int nb,
                                                  unsigned int* counter, double* out) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == (unsigned)nb - 1u;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < 32) {
    const volatile double* p = partial;
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) v += p[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) {
      *out = v;
      *counter = 0u;
    }
  }
}

// The same for K outputs at once: out[k] = sum of partial[k * nb .. k * nb + nb).
__device__ __forceinline__ void last_block_reduce_k(const double* __restrict__ partial, int nb,
                                                    int K, unsigned int* counter, double* out) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == (unsigned)nb - 1u;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = w; k < K; k += blockDim.x >> 5) {
    const volatile double* p = partial + (int64_t)k * nb;
    double v = 0.0;
    for (int b = lane; b < nb; b += 32) v += p[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) out[k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
}

// partial[i*gridDim.x + b] = block b's share of A_i . bvec (grid.y = vector i).
// FP32 x FP32 products are summed in FP32 over groups of four strided elements and
// the group sums in FP64; every other combination is formed and summed in FP64.
template <typename TA, typename TB>
__global__ void __launch_bounds__(kRedThreads) k_dots(const TA* __restrict__ A, int64_t lda,
                                                      const TB* __restrict__ b, int64_t N,
                                                      double* __restrict__ partial,
                                                      unsigned int* counters, double* out) {
  const int i = blockIdx.y;
  const TA* __restrict__ a = A + (int64_t)i * lda;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc = 0.0;
  if constexpr (std::is_same<TA, float>::value && std::is_same<TB, float>::value) {
    for (; j + 3 * stride < N; j += 4 * stride) {
      float p = a[j] * b[j];
      p = fmaf(a[j + stride], b[j + stride], p);
      p = fmaf(a[j + 2 * stride], b[j + 2 * stride], p);
      p = fmaf(a[j + 3 * stride], b[j + 3 * stride], p);
      acc += (double)p;
    }
  }
  for (; j < N; j += stride) acc += (double)a[j] * (double)b[j];
  __shared__ double red[kRedThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) v += red[w];
    partial[(int64_t)i * gridDim.x + blockIdx.x] = v;
  }
  if (counters)
    last_block_reduce(partial + (int64_t)i * gridDim.x, gridDim.x, counters + i, out + i);
}

// Two products per vector in one pass over A: partial[i*gridDim.x + b] = block b's
// share of A_i . b1 and partial[(gridDim.y + i)*gridDim.x + b] that of A_i . b2
// (same arithmetic as k_dots).
template <typename TA, typename TB>
__global__ void __launch_bounds__(kRedThreads) k_dots2(const TA* __restrict__ A, int64_t lda,
                                                       const TB* __restrict__ b1,
                                                       const TB* __restrict__ b2, int64_t N,
                                                       double* __restrict__ partial,
                                                       unsigned int* counters, double* out1,
                                                       double* out2) {
  const int i = blockIdx.y;
  const TA* __restrict__ a = A + (int64_t)i * lda;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc1 = 0.0, acc2 = 0.0;
  if constexpr (std::is_same<TA, float>::value && std::is_same<TB, float>::value) {
    for (; j + 3 * stride < N; j += 4 * stride) {
      const float a0 = a[j], a1 = a[j + stride], a2 = a[j + 2 * stride], a3 = a[j + 3 * stride];
      float p = a0 * b1[j], q = a0 * b2[j];
      p = fmaf(a1, b1[j + stride], p);
      q = fmaf(a1, b2[j + stride], q);
      p = fmaf(a2, b1[j + 2 * stride], p);
      q = fmaf(a2, b2[j + 2 * stride], q);
      p = fmaf(a3, b1[j + 3 * stride], p);
      q = fmaf(a3, b2[j + 3 * stride], q);
      acc1 += (double)p;
      acc2 += (double)q;
    }
  }
  for (; j < N; j += stride) {
    const double av = (double)a[j];
    acc1 += av * (double)b1[j];
    acc2 += av * (double)b2[j];
  }
  __shared__ double red[2][kRedThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc1 += __shfl_down_sync(0xffffffffu, acc1, o);
    acc2 += __shfl_down_sync(0xffffffffu, acc2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = acc1;
    red[1][threadIdx.x >> 5] = acc2;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double v = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) v += red[threadIdx.x][w];
    partial[((int64_t)threadIdx.x * gridDim.y + i) * gridDim.x + blockIdx.x] = v;
  }
  // one counter per vector: the last block sums both outputs of vector i
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counters + i, 1u) == gridDim.x - 1u;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < 64) {
    const int which = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const volatile double* p = partial + ((int64_t)which * gridDim.y + i) * gridDim.x;
    double v = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) v += p[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) (which ? out2 : out1)[i] = v;
  }
  if (threadIdx.x == 0) counters[i] = 0u;
}


// out (FP64) = (mode 0: 0, 1: out, -1: out) +/- sum_i coef[i] * A_i.  For FP32 A the
// combination is formed in FP32 (it is a correction whose rounding is relative to
// itself) and added to out in FP64.
template <typename TA>
__global__ void k_lincomb(double* __restrict__ out, const TA* __restrict__ A, int64_t lda, int m,
                          const double* __restrict__ coef, int64_t N, int mode) {
  __shared__ double c[kMaxSub];
  if (threadIdx.x < m) c[threadIdx.x] = coef[threadIdx.x];
  __syncthreads();
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    double v;
    if constexpr (std::is_same<TA, float>::value) {
      float f = 0.0f;
      int i = 0;
      for (; i + 4 <= m; i += 4) {
        const float a0 = A[i * lda + j], a1 = A[(i + 1) * lda + j];
        const float a2 = A[(i + 2) * lda + j], a3 = A[(i + 3) * lda + j];
        f = fmaf((float)c[i], a0, f);
        f = fmaf((float)c[i + 1], a1, f);
        f = fmaf((float)c[i + 2], a2, f);
        f = fmaf((float)c[i + 3], a3, f);
      }
      for (; i < m; ++i) f = fmaf((float)c[i], A[i * lda + j], f);
      v = (double)f;
    } else {
      v = 0.0;
      for (int i = 0; i < m; ++i) v += c[i] * A[i * lda + j];
    }
    if (mode == 0) out[j] = v;
    else if (mode > 0) out[j] += v;
    else out[j] -= v;
  }
}

// FP32 out = out - sum_i coef[i] * A_i (FP32 arithmetic)
__global__ void k_lincomb_sub_f32(float* __restrict__ out, const float* __restrict__ A,
                                  int64_t lda, int m, const double* __restrict__ coef, int64_t N) {
  __shared__ float c[kMaxSub];
  if (threadIdx.x < m) c[threadIdx.x] = (float)coef[threadIdx.x];
  __syncthreads();
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    float f = out[j];
    int i = 0;
    for (; i + 4 <= m; i += 4) {
      const float a0 = A[i * lda + j], a1 = A[(i + 1) * lda + j];
      const float a2 = A[(i + 2) * lda + j], a3 = A[(i + 3) * lda + j];
      f = fmaf(-c[i], a0, f);
      f = fmaf(-c[i + 1], a1, f);
      f = fmaf(-c[i + 2], a2, f);
      f = fmaf(-c[i + 3], a3, f);
    }
    for (; i < m; ++i) f = fmaf(-c[i], A[i * lda + j], f);
    out[j] = f;
  }
}

// y = x / sqrt(nrm2[0]) with type conversion
template <typename TI, typename TO>
__global__ void k_scale_store(const TI* __restrict__ x, const double* __restrict__ nrm2,
                              TO* __restrict__ y, int64_t N) {
  if constexpr (std::is_same<TI, float>::value) {
    const float s = (float)(1.0 / sqrt(nrm2[0]));
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
         j += (int64_t)gridDim.x * blockDim.x)
      y[j] = (TO)(x[j] * s);
  } else {
    const double s = 1.0 / sqrt(nrm2[0]);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
         j += (int64_t)gridDim.x * blockDim.x)
      y[j] = (TO)(x[j] * s);
  }
}

// Residual and preconditioned correction.
//   r = y0*s0 + sum_i y[i] W_i - theta*(y0*x0 + sum_i y[i] V_i)
//   t = r / floor(D - theta);  partial ||r||^2 per block
// (x0, s0 may be NULL; then y0 is ignored.)  For FP32 V, W the two sums over i
// are formed in FP32: they carry the correction, whose rounding is relative to
// itself, while the FP64 parts y0*s0 and y0*x0 stay FP64.
template <typename TV>
__global__ void __launch_bounds__(kRedThreads) k_residual(
    const double* __restrict__ x0, const double* __restrict__ s0, const TV* __restrict__ V,
    const TV* __restrict__ W, int64_t ld, int m, const double* __restrict__ ritz, /* [0]=theta, [1..]=y */
    int has_x0, const double* __restrict__ D, double floor_, int64_t N, double* __restrict__ t,
    double* __restrict__ partial, unsigned int* counter = nullptr, double* rr_out = nullptr) {
  __shared__ double y[kMaxSub + 1];
  __shared__ float yf[kMaxSub + 1];
  __shared__ double red[kRedThreads / 32];
  if (threadIdx.x <= m + has_x0) {
    y[threadIdx.x] = ritz[1 + threadIdx.x];
    yf[threadIdx.x] = (float)ritz[1 + threadIdx.x];
  }
  __syncthreads();
  const double theta = ritz[0];
  const int o = has_x0 ? 1 : 0;
  double acc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    double hx = 0.0, xx = 0.0;
    if (has_x0) {
      hx = y[0] * s0[j];
      xx = y[0] * x0[j];
    }
    if constexpr (std::is_same<TV, float>::value) {
      float hf = 0.0f, xf = 0.0f;
      int i = 0;
      for (; i + 4 <= m; i += 4) {  // eight loads in flight
        float w4[4], v4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          w4[u] = W[(i + u) * ld + j];
          v4[u] = V[(i + u) * ld + j];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float yi = yf[o + i + u];
          hf = fmaf(yi, w4[u], hf);
          xf = fmaf(yi, v4[u], xf);
        }
      }
      for (; i < m; ++i) {
        const float yi = yf[o + i];
        hf = fmaf(yi, W[i * ld + j], hf);
        xf = fmaf(yi, V[i * ld + j], xf);
      }
      hx += (double)hf;
      xx += (double)xf;
    } else {
      for (int i = 0; i < m; ++i) {
        hx += y[o + i] * W[i * ld + j];
        xx += y[o + i] * V[i * ld + j];
      }
    }
    const double r = hx - theta * xx;
    acc += r * r;
    // the correction only steers the search: divide in FP32
    float den = (float)(D[j] - theta);
    const float fl = (float)floor_;
    if (fabsf(den) < fl) den = (den < 0.0f) ? -fl : fl;
    t[j] = (double)__fdividef((float)r, den);
  }
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o2);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) v += red[w];
    partial[blockIdx.x] = v;
  }
  if (counter) last_block_reduce(partial, gridDim.x, counter, rr_out);
}

// ------------------------------------------- mixed inner iteration, FP32 --
//
// FP64 arithmetic runs at a small fraction of the FP32 rate on this part, so the
// passes of the mixed inner iteration do no FP64 arithmetic per element: the anchor
// enters through x32 = fp32(x) and the FP32 anchor residual ra = fp32(s - theta_a x)
// (theta_a = x.s), whose rounding is relative to the residual itself, and the
// coupling to the anchor is G_0i = theta_a S_0i + ra.v_i with the same S_0i = x32.v_i
// that goes into S, so the pencil stays consistent.  MB bounds the number of basis
// vectors a pass reads (a register array).

constexpr int kVecGrid = 4 * kNumSMs;  // blocks of the fused vector passes
constexpr int kVecOut = 2 * kMaxSub + 4;  // dot products one fused pass can return
// per-block partial sums: the dot kernels and the fused passes
constexpr int kPartial = std::max(2 * kRedGrid * (kMaxSub + 1), kVecOut * kVecGrid);

// K running sums of one thread (FP32: a thread sums N / (kVecGrid * 256) products, a
// relative error far below what the inner iteration needs, whose pencil and
// directions already carry the FP32 / BF16 rounding of the products), combined in
// FP64 across threads and blocks.
template <int K>
struct Sums {
  float f[K];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < K; ++k) f[k] = 0.f;
  }
  // Block sums into partial[slot * gridDim.x + blockIdx.x], then the last block writes
  // out[slot]: sums 0 .. nA-1 go to slots 0 .. nA-1, sums offB .. offB+nB-1 to slots
  // nA .. nA+nB-1 (the sums stay in registers: every index into f is a constant).
  __device__ __forceinline__ void finish(int nA, int offB, int nB, double* __restrict__ partial,
                                         unsigned int* counter, double* out) {
    __shared__ double red[kVecOut][kRedThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int slot = k < nA ? k : (k >= offB && k < offB + nB) ? nA + k - offB : -1;
      if (slot < 0) continue;  // uniform over the block
      double v = (double)f[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[slot][w] = v;
    }
    __syncthreads();
    const int n = nA + nB;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      double v = 0.0;
      for (int q = 0; q < kRedThreads / 32; ++q) v += red[k][q];
      partial[(int64_t)k * gridDim.x + blockIdx.x] = v;
    }
    last_block_reduce_k(partial, gridDim.x, n, counter, out);
  }
};

// The inner residual and its correction, with the dot products the orthogonalisation
// needs:  u = y0 x + V y,  r = y0 ra + y0 (theta_a - theta) x32 + W y - theta V y,
// t = r / floor(D32 - theta);  out = {r.r, t.t, x32.t, V_i.t (i < m)}.
template <int MB>
__global__ void __launch_bounds__(kRedThreads) k_res32(
    const float* __restrict__ ra, const float* __restrict__ x32, const float* __restrict__ V,
    const float* __restrict__ W, int64_t ld, int m, const double* __restrict__ ritz,
    const double* __restrict__ theta_a, const float* __restrict__ D32, float floor_, int64_t N,
    float* __restrict__ t, double* __restrict__ partial, unsigned int* counter,
    double* __restrict__ out) {
  __shared__ float y[kMaxSub + 1];
  if (threadIdx.x <= m) y[threadIdx.x] = (float)ritz[1 + threadIdx.x];
  __syncthreads();
  const float theta = (float)ritz[0];
  const float y0 = y[0], a0 = (float)((*theta_a - ritz[0]) * ritz[1]);
  Sums<MB + 3> acc;
  acc.zero();
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    float v[MB];
    float hv = 0.f, xv = 0.f;
#pragma unroll
    for (int i = 0; i < MB; ++i) {
      v[i] = 0.f;
      if (i < m) {
        v[i] = V[i * ld + j];
        hv = fmaf(y[1 + i], W[i * ld + j], hv);
        xv = fmaf(y[1 + i], v[i], xv);
      }
    }
    const float xj = x32[j];
    const float r = fmaf(y0, ra[j], fmaf(a0, xj, fmaf(-theta, xv, hv)));
    float den = D32[j] - theta;
    if (fabsf(den) < floor_) den = (den < 0.0f) ? -floor_ : floor_;
    const float tj = __fdividef(r, den);
    t[j] = tj;
    acc.f[0] = fmaf(r, r, acc.f[0]);
    acc.f[1] = fmaf(tj, tj, acc.f[1]);
    acc.f[2] = fmaf(xj, tj, acc.f[2]);
#pragma unroll
    for (int i = 0; i < MB; ++i) acc.f[3 + i] = fmaf(v[i], tj, acc.f[3 + i]);
  }
  acc.finish(m + 3, 0, 0, partial, counter, out);
}

// Coefficients of one Gram-Schmidt pass, passed by value (no host-to-device copy).
struct OrthoCoef {
  float c[kMaxSub + 1];  // c[0] for x32, c[1 + i] for V_i
  float scale;
};

// o = (t - c0 x32 - sum_i c_i V_i) * scale (o may be t); out = {x32.o, V_i.o (i < m), o.o}.
template <int MB>
__global__ void __launch_bounds__(kRedThreads) k_ortho32(
    const float* t, const float* __restrict__ x32, const float* __restrict__ V,
    int64_t ld, int m, const OrthoCoef cf, float* o, int64_t N,
    double* __restrict__ partial, unsigned int* counter, double* __restrict__ out) {
  Sums<MB + 2> acc;
  acc.zero();
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    float v[MB];
    const float xj = x32[j];
    float p = fmaf(-cf.c[0], xj, t[j]);
#pragma unroll
    for (int i = 0; i < MB; ++i) {
      v[i] = 0.f;
      if (i < m) {
        v[i] = V[i * ld + j];
        p = fmaf(-cf.c[1 + i], v[i], p);
      }
    }
    p *= cf.scale;
    o[j] = p;
    acc.f[0] = fmaf(xj, p, acc.f[0]);
#pragma unroll
    for (int i = 0; i < MB; ++i) acc.f[1 + i] = fmaf(v[i], p, acc.f[1 + i]);
    acc.f[MB + 1] = fmaf(p, p, acc.f[MB + 1]);
  }
  acc.finish(m + 1, MB + 1, 1, partial, counter, out);  // the norm lands in out[m + 1]
}

// The pencil column of a new vector v = V_j with product w = W_j:
// out = {x32.v, ra.v, V_i.w (i <= j), V_i.v (i <= j)}.
template <int MB>
__global__ void __launch_bounds__(kRedThreads) k_col32(
    const float* __restrict__ x32, const float* __restrict__ ra, const float* __restrict__ V,
    const float* __restrict__ W, int64_t ld, int j, int64_t N, double* __restrict__ partial,
    unsigned int* counter, double* __restrict__ out) {
  Sums<2 * MB + 2> acc;
  acc.zero();
  const int n = j + 1;  // vectors V_0 .. V_j
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float vj = V[j * ld + e], wj = W[j * ld + e];
    acc.f[0] = fmaf(x32[e], vj, acc.f[0]);
    acc.f[1] = fmaf(ra[e], vj, acc.f[1]);
#pragma unroll
    for (int i = 0; i < MB; ++i) {
      if (i < n) {
        const float vi = V[i * ld + e];
        acc.f[2 + i] = fmaf(vi, wj, acc.f[2 + i]);
        acc.f[2 + MB + i] = fmaf(vi, vj, acc.f[2 + MB + i]);
      }
    }
  }
  acc.finish(2 + n, 2 + MB, n, partial, counter, out);  // {x.v, ra.v, V.w[0..n), V.v[0..n)}
}

// The anchor row of the pencil for the kept vectors V_0 .. V_{m-1}:
// out = {x32.V_i (i < m), ra.V_i (i < m)}.
template <int MB>
__global__ void __launch_bounds__(kRedThreads) k_anchor_row32(
    const float* __restrict__ x32, const float* __restrict__ ra, const float* __restrict__ V,
    int64_t ld, int m, int64_t N, double* __restrict__ partial, unsigned int* counter,
    double* __restrict__ out) {
  Sums<2 * MB> acc;
  acc.zero();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float xe = x32[e], re = ra[e];
#pragma unroll
    for (int i = 0; i < MB; ++i) {
      if (i < m) {
        const float vi = V[i * ld + e];
        acc.f[i] = fmaf(xe, vi, acc.f[i]);
        acc.f[MB + i] = fmaf(re, vi, acc.f[MB + i]);
      }
    }
  }
  acc.finish(m, MB, m, partial, counter, out);  // {x32.V_i, ra.V_i}
}

// A restart of the mixed solver in one pass over {x, s, V, W}: for the kk lowest Ritz
// vectors y_k of the pencil (anchor coefficient y_k0, V coefficients y_ki),
//   k = 0:  xn = y_00 x + sum_i y_0i V_i,  sxn = y_00 s + sum_i y_0i W_i   (FP64 out)
//   k >= 1: U_{k-1} = y_k0 x32 + sum_i y_ki V_i,
//           WU_{k-1} = y_k0 (ra + theta_a x32) + sum_i y_ki W_i          (FP32 out)
// (s = ra + theta_a x up to the FP32 rounding of ra and x32).  The V and W sums are FP32,
// the corrections they carry; only xn and sxn take FP64 arithmetic.
template <int MB>
__global__ void __launch_bounds__(kRedThreads) k_restart32(
    const double* __restrict__ x, const double* __restrict__ sx, const float* __restrict__ x32,
    const float* __restrict__ ra, const float* __restrict__ V, const float* __restrict__ W,
    int64_t ld, int m, const double* __restrict__ all, int kk, const double* __restrict__ theta_a,
    int64_t N, double* __restrict__ xn, double* __restrict__ sxn, float* __restrict__ U,
    float* __restrict__ WU) {
  __shared__ float yv[kMaxSub][kMaxSub];
  __shared__ double y0[kMaxSub];
  for (int t = threadIdx.x; t < kMaxSub * kMaxSub; t += blockDim.x) yv[t / kMaxSub][t % kMaxSub] = 0.f;
  __syncthreads();
  for (int t = threadIdx.x; t < kk * (m + 1); t += blockDim.x) {
    const int k = t / (m + 1), i = t % (m + 1);
    const double v = all[(size_t)k * kRitzStride + 1 + i];
    if (i == 0) y0[k] = v;
    else yv[k][i - 1] = (float)v;
  }
  __syncthreads();
  const float tha = (float)*theta_a;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    float v[MB], w[MB];
#pragma unroll
    for (int i = 0; i < MB; ++i) {
      v[i] = 0.f, w[i] = 0.f;
      if (i < m) v[i] = V[i * ld + j], w[i] = W[i * ld + j];
    }
    const float xf = x32[j], sf = fmaf(tha, xf, ra[j]);
    for (int k = 0; k < kk; ++k) {
      float a = 0.f, b = 0.f;
#pragma unroll
      for (int i = 0; i < MB; ++i) a = fmaf(yv[k][i], v[i], a), b = fmaf(yv[k][i], w[i], b);
      if (k == 0) {
        xn[j] = fma(y0[0], x[j], (double)a);
        sxn[j] = fma(y0[0], sx[j], (double)b);
      } else {
        const float yk = (float)y0[k];
        U[(k - 1) * ld + j] = fmaf(yk, xf, a);
        WU[(k - 1) * ld + j] = fmaf(yk, sf, b);
      }
    }
  }
}

// x32 = fp32(x), ra = fp32(s - theta_a x) with theta_a = G00 / S00 (written to *theta_a)
__global__ void k_anchor32(const double* __restrict__ x, const double* __restrict__ s,
                           const double* __restrict__ gs, double* __restrict__ theta_a,
                           float* __restrict__ x32, float* __restrict__ ra, int64_t N) {
  const double th = gs[0] / gs[1];
  if (blockIdx.x == 0 && threadIdx.x == 0) *theta_a = th;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    const double xj = x[j];
    x32[j] = (float)xj;
    ra[j] = (float)fma(-th, xj, s[j]);
  }
}

// G, S entries of column col from a k_col32 result (n = col vectors before the anchor
// offset): G[0][col] = theta_a x.v + ra.v, S[0][col] = x.v, G[i+1][col] = V_i.w,
// S[i+1][col] = V_i.v (symmetric)
__global__ void k_set_col32(double* G, double* S, int ldg, int col, const double* sums, int n,
                            const double* theta_a) {
  const int i = threadIdx.x;
  if (i == 0) {
    const double g = *theta_a * sums[0] + sums[1];
    G[col] = g, G[col * ldg] = g;
    S[col] = sums[0], S[col * ldg] = sums[0];
  } else if (i <= n) {
    const double g = sums[1 + i], sv = sums[1 + n + i];
    G[i * ldg + col] = g, G[col * ldg + i] = g;
    S[i * ldg + col] = sv, S[col * ldg + i] = sv;
  }
}

// Row 0 of (G, S) for the kept vectors from a k_anchor_row32 result
__global__ void k_set_row32(double* G, double* S, int ldg, const double* sums, int m,
                            const double* theta_a) {
  const int i = threadIdx.x;
  if (i < m) {
    const double sv = sums[i], g = *theta_a * sv + sums[m + i];
    G[1 + i] = g, G[(1 + i) * ldg] = g;
    S[1 + i] = sv, S[(1 + i) * ldg] = sv;
  }
}

// 1/sqrt(x) for x > 0 to FP64 accuracy: an FP32 estimate refined by two Newton steps
// (each roughly squares the relative error), which keeps FP64 division and square root
// (long instruction sequences on this part's FP64 pipe) out of the serial chains below.
__device__ __forceinline__ double rsqrt64(double x) {
  const float xf = (float)x;
  if (!(xf > 1e-30f && xf < 1e30f)) return 1.0 / sqrt(x);
  double y = (double)rsqrtf(xf);
  y = y * fma(-0.5 * x * y, y, 1.5);
  y = y * fma(-0.5 * x * y, y, 1.5);
  return y;
}

__device__ __forceinline__ double warp_sum64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;  // the same in every lane (each butterfly step adds the same two terms)
}

// Rotation (c, s) that zeroes A_pq of the symmetric 2 x 2 block (app, apq; apq, aqq):
// t = tan(angle) from tau = (aqq - app) / (2 apq), the root of t^2 + 2 tau t - 1 = 0 of
// smaller magnitude, c = 1 / sqrt(1 + t^2), s = t c.  In FP64 the tangent is formed in
// FP32 and the cosine refined by Newton steps on 1 / sqrt(1 + t^2), so the rotation is
// orthogonal to FP64 rounding (a rotation that zeroes A_pq only to FP32 accuracy is
// still a valid Jacobi rotation; later sweeps remove the remainder).
__device__ __forceinline__ void jacobi_rotation(float app, float aqq, float apq, float& c,
                                                float& s) {
  // approximate division and square root: the rotation only has to be orthogonal, which
  // c = 1 / sqrt(1 + t^2), s = t c is for any t, to FP32 rounding
  const float tau = __fdividef(aqq - app, 2.0f * apq);
  float t = 0.0f;  // tau not finite: A_pq is negligible, no rotation
  if (fabsf(tau) < 1e18f) {
    const float x = fmaf(tau, tau, 1.0f);
    t = __fdividef(tau >= 0.0f ? 1.0f : -1.0f, fabsf(tau) + x * rsqrtf(x));
  } else if (isfinite(tau)) {
    t = __fdividef(0.5f, tau);
  }
  c = rsqrtf(fmaf(t, t, 1.0f));
  s = t * c;
}
__device__ __forceinline__ void jacobi_rotation(double app, double aqq, double apq, double& c,
                                                double& s) {
  const float tau = (float)(aqq - app) / (2.0f * (float)apq);
  float tf = 0.0f;
  if (isfinite(tau))
    tf = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
  const double t = (double)tf, x = fma(t, t, 1.0);
  double y = (double)rsqrtf((float)x);
  y = y * fma(-0.5 * x * y, y, 1.5);
  y = y * fma(-0.5 * x * y, y, 1.5);
  c = y;
  s = t * y;
}

template <typename T>
struct JacobiFloor;
template <>
struct JacobiFloor<float> {  // eps = 2^-24
  static constexpr double eps2 = 3.5527136788005009e-15, stall = 1e-10;
};
template <>
struct JacobiFloor<double> {  // eps = 2^-53
  static constexpr double eps2 = 1.2325951644078310e-32, stall = 1e-24;
};

// Cyclic Jacobi on the symmetric mm x mm matrix A (m real rows, mm = m rounded up to
// even; a padding row is isolated with a huge diagonal), round-robin parallel ordering
// in one block of kRRThreads threads, rotations accumulated into Q.  Converged when the
// off-diagonal mass of the m x m block is at the rounding floor of the rotations,
// (4 m eps)^2 relative to the diagonal's, or stops falling near it; 30 sweeps at most.
// The pairing is the round-robin tournament in closed form: at step t position 0 holds
// index 0 and position k >= 1 holds 1 + ((k - 1 - t) mod (mm - 1)), and position k meets
// position mm - 1 - k; each step moves the index at a position k >= 1 one down (1 wraps
// to mm - 1).  In the updates thread (w, l) takes row or column l of the pairs w, w + 4,
// ...  cs holds mm/2 (c, s) pairs of T, pr is int scratch, red2 [4][2] of T.
template <typename T>
__device__ void jacobi_sweeps(T (*A)[kMaxSub + 1], T (*Q)[kMaxSub + 1], int m, int mm, T* cs,
                              int (*pr)[2], T (*red2)[2]) {
  const int lane = threadIdx.x, w = lane >> 5, l = lane & 31;
  constexpr int kW = kRRThreads / 32;
  const int h = mm / 2, nm = mm - 1;
  const T floor_rel = (T)(16.0 * (double)m * (double)m * JacobiFloor<T>::eps2);
  const T stall = (T)JacobiFloor<T>::stall;
  T prev_off = 0;
  for (int sweep = 0; sweep < 30; ++sweep) {
    T off = 0, dia = 0;
    for (int r = w; r < m; r += kW)
      if (l < m) {
        const T v = A[r][l];
        if (r != l) off += v * v;
        else dia += v * v;
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if (l == 0) {
      red2[w][0] = off;
      red2[w][1] = dia;
    }
    __syncthreads();
    off = 0;
    dia = 0;
    for (int k = 0; k < kW; ++k) {
      off += red2[k][0];
      dia += red2[k][1];
    }
    __syncthreads();
    if (off <= floor_rel * dia || off == (T)0) break;
    if (sweep > 0 && off >= (T)0.25 * prev_off && off <= stall * dia) break;
    prev_off = off;
    int a = lane, b = mm - 1 - lane;  // indices at positions lane and mm - 1 - lane
    for (int step = 0; step < nm; ++step) {
      if (lane < h) {
        const int p = min(a, b), q = max(a, b);
        pr[lane][0] = p;
        pr[lane][1] = q;
        const T apq = A[p][q];
        T c = 1, sn = 0;
        if (apq != (T)0 && p < m && q < m) jacobi_rotation(A[p][p], A[q][q], apq, c, sn);
        cs[2 * lane] = c;
        cs[2 * lane + 1] = sn;
        if (a != 0) a = a == 1 ? nm : a - 1;
        b = b == 1 ? nm : b - 1;
      }
      __syncthreads();
      if (l < mm)  // A <- J^T A (rows p, q), column l
        for (int k = w; k < h; k += kW) {
          const int p = pr[k][0], q = pr[k][1];
          const T c = cs[2 * k], sn = cs[2 * k + 1];
          const T ap = A[p][l], aq = A[q][l];
          A[p][l] = c * ap - sn * aq;
          A[q][l] = sn * ap + c * aq;
        }
      __syncthreads();
      if (l < mm)  // A <- A J, Q <- Q J (cols p, q), row l
        for (int k = w; k < h; k += kW) {
          const int p = pr[k][0], q = pr[k][1];
          const T c = cs[2 * k], sn = cs[2 * k + 1];
          const T ap = A[l][p], aq = A[l][q];
          A[l][p] = c * ap - sn * aq;
          A[l][q] = sn * ap + c * aq;
          const T qp = Q[l][p], qq = Q[l][q];
          Q[l][p] = c * qp - sn * qq;
          Q[l][q] = sn * qp + c * qq;
        }
      __syncthreads();
    }
  }
}

// Lowest eigenpair of the symmetric m x m pencil (G, S) (row-major, leading dim ldg;
// S == NULL means S = I), in one block of kRRThreads threads (m <= kMaxSub).  FP64 runs
// at a small fraction of the FP32 rate on this part, so the FP64 work is kept to what
// fixes the result's accuracy:
//   1. The pencil is reduced to a symmetric C with a factor M, M^T S M = I, C = M^T G M:
//      near the identity (m max|S - I| <= 1e-4) M = S^-1/2 by its series; otherwise the
//      Cholesky factor S = L L^T (FP64, right-looking, the pivots' 1/sqrt by rsqrt64),
//      M = L^-T; without S, C = (G + G^T) / 2.
//   2. Cyclic Jacobi on fp32(C) in FP32 (warm-started, when the pencil grew
//      by one row and column since the last call, from the previous eigenvectors in
//      qkeep: the transformed matrix is then diagonal but for its last row and column,
//      up to FP32 rounding).
//   3. The lowest pair refined in FP64 against C: with r = C z - theta z and
//      theta = z^T C z (|z| = 1), z <- z - sum_{j != 0} q_j (q_j^T r) / (lambda_j - theta)
//      over the FP32 eigenpairs (q_j, lambda_j), the Newton correction for an eigenvector
//      with the FP32 spectral inverse of C - theta on the complement of q_0, until |r| is
//      at the rounding floor (16 m eps64 max|lambda|); each step gains about the FP32
//      accuracy times the spectral spread over the gap.
//   4. If the two lowest FP32 eigenvalues are closer than 1e-5 of the spectral scale, or
//      the refinement does not reach the floor in 8 steps, FP64 Jacobi on C instead (the
//      rotations' tangents in FP32, cosines refined to FP64).
// Eigenvectors are mapped back, y = M z, so that y^T S y = 1.  out[0] = theta,
// out[1..m] = y (largest |component| > 0).  If all != NULL every eigenpair is written in
// ascending order, all[j * kRitzStride] = lambda_j, all[j * kRitzStride + 1 ..] = y_j
// (pairs other than the lowest to the FP32 solve's accuracy when it was kept).  path
// (optional): bit 0 the series factor, bit 1 the Cholesky factor, bit 2 the refined FP32
// solve (else FP64 Jacobi).
__global__ void __launch_bounds__(kRRThreads) k_rr(const double* __restrict__ G, int ldg, int m,
                                           double* __restrict__ out,
                                           const double* __restrict__ S,
                                           double* __restrict__ all = nullptr,
                                           double* __restrict__ qkeep = nullptr, int warm = 0,
                                           int* __restrict__ path = nullptr) {
  __shared__ double Cm[kMaxSub][kMaxSub + 1];  // the reduced matrix C (FP64)
  __shared__ double L[kMaxSub][kMaxSub + 1];   // Cholesky factor of S
  __shared__ double X[kMaxSub][kMaxSub + 1];   // scratch; A of the FP64 fallback
  __shared__ double U[kMaxSub][kMaxSub + 1];   // Q of the FP64 fallback, or A32 | Q32
  __shared__ double Linv[kMaxSub];
  __shared__ double z[kMaxSub];
  __shared__ double part[kRRThreads / 32][kMaxSub];
  __shared__ double cs64[kMaxSub];
  __shared__ double red64[kRRThreads / 32][2];
  __shared__ float lam[kMaxSub];
  __shared__ float rbuf[kMaxSub];
  __shared__ float pbuf[kMaxSub];
  __shared__ int pr[kMaxSub / 2][2];
  __shared__ int rank_of[kMaxSub];
  __shared__ int s_flag;
  __shared__ int s_emax;
  __shared__ double s_theta;
  float (*A32)[kMaxSub + 1] = reinterpret_cast<float (*)[kMaxSub + 1]>(&U[0][0]);
  float (*Q32)[kMaxSub + 1] = A32 + kMaxSub;
  float (*T32)[kMaxSub + 1] = reinterpret_cast<float (*)[kMaxSub + 1]>(&X[0][0]);
  const int lane = threadIdx.x;  // thread index in the block
  const int w = lane >> 5, l = lane & 31;
  const unsigned full = 0xffffffffu;
  const int mm = m + (m & 1);  // even size for the tournament; the pad row/col is isolated

  // ---- 1. C (FP64)
  bool use_s = false, use_m = false;
  if (S) {
    // E = S - I.  Near the identity (a basis orthonormal up to FP32 rounding, as the
    // mixed solver's), the symmetric factor M = S^-1/2 = I - E/2 + 3E^2/8 - 5E^3/16 +
    // O(E^4) (exact to FP64 rounding while m max|E_ij| <= 1e-4) takes the Cholesky
    // factor's place: C = M G M and y = M z, from small matrix products that every
    // thread shares, instead of m serial pivots and triangular solves.
    if (lane == 0) s_emax = 0;
    __syncthreads();
    float e = 0.0f;
    for (int i = lane; i < m * m; i += kRRThreads) {
      const int r = i / m, c = i % m;
      const double v = 0.5 * (S[r * ldg + c] + S[c * ldg + r]) - (r == c ? 1.0 : 0.0);
      X[r][c] = v;
      Cm[r][c] = 0.5 * (G[r * ldg + c] + G[c * ldg + r]);
      e = fmaxf(e, fabsf((float)v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = fmaxf(e, __shfl_xor_sync(full, e, o));
    if (l == 0) atomicMax(&s_emax, __float_as_int(e));  // non-negative: ordered as integers
    __syncthreads();
    use_m = (float)m * __int_as_float(s_emax) <= 1e-4f;
  }
  if (use_m) {
    for (int i = lane; i < m * m; i += kRRThreads) {  // U = E^2
      const int r = i / m, c = i % m;
      double v = 0.0;
      for (int k = 0; k < m; ++k) v = fma(X[r][k], X[k][c], v);
      U[r][c] = v;
    }
    __syncthreads();
    for (int i = lane; i < m * m; i += kRRThreads) {  // L = M
      const int r = i / m, c = i % m;
      double v = 0.0;
      for (int k = 0; k < m; ++k) v = fma(X[r][k], U[k][c], v);
      L[r][c] = (r == c ? 1.0 : 0.0) - 0.5 * X[r][c] + 0.375 * U[r][c] - 0.3125 * v;
    }
    __syncthreads();
    for (int i = lane; i < m * m; i += kRRThreads) {  // U = G M
      const int r = i / m, c = i % m;
      double v = 0.0;
      for (int k = 0; k < m; ++k) v = fma(Cm[r][k], L[k][c], v);
      U[r][c] = v;
    }
    __syncthreads();
    for (int i = lane; i < m * m; i += kRRThreads) {  // X = M G M
      const int r = i / m, c = i % m;
      double v = 0.0;
      for (int k = 0; k < m; ++k) v = fma(L[r][k], U[k][c], v);
      X[r][c] = v;
    }
    __syncthreads();
    for (int i = lane; i < m * m; i += kRRThreads) {
      const int r = i / m, c = i % m;
      Cm[r][c] = 0.5 * (X[r][c] + X[c][r]);
    }
  } else if (S) {
    for (int i = lane; i < m * m; i += kRRThreads) {
      const int r = i / m, c = i % m;
      if (c <= r) L[r][c] = 0.5 * (S[r * ldg + c] + S[c * ldg + r]);
    }
    __syncthreads();
    use_s = true;
    for (int j = 0; j < m; ++j) {
      const double d = L[j][j];  // the same in every thread
      if (!(d > 0.0)) {
        use_s = false;
        break;
      }
      const double inv = rsqrt64(d);
      for (int i = j + 1 + lane; i < m; i += kRRThreads) L[i][j] *= inv;
      __syncthreads();
      const int r = m - j - 1;  // trailing block rows j+1..m-1
      for (int t = lane; t < r * r; t += kRRThreads) {
        const int i = j + 1 + t / r, k = j + 1 + t % r;
        if (k <= i) L[i][k] -= L[i][j] * L[k][j];
      }
      if (lane == 0) {
        Linv[j] = inv;
        L[j][j] = d * inv;
      }
      __syncthreads();
    }
  }
  // columns spread over the four warps: thread (w, l) takes column 4 l + w
  const int my_col = 4 * l + w;
  if (use_s) {
    // X = L^-1 Gs, then C = L^-1 X^T, column by column (forward substitution)
    if (my_col < m) {
      for (int i = 0; i < m; ++i) {
        double v = 0.5 * (G[i * ldg + my_col] + G[my_col * ldg + i]);
        for (int k = 0; k < i; ++k) v -= L[i][k] * X[k][my_col];
        X[i][my_col] = v * Linv[i];
      }
    }
    __syncthreads();
    if (my_col < m) {
      for (int i = 0; i < m; ++i) {
        double v = X[my_col][i];
        for (int k = 0; k < i; ++k) v -= L[i][k] * Cm[k][my_col];
        Cm[i][my_col] = v * Linv[i];
      }
    }
    __syncthreads();
    for (int i = lane; i < m * m; i += kRRThreads) {
      const int r = i / m, c = i % m;
      if (c < r) {
        const double v = 0.5 * (Cm[r][c] + Cm[c][r]);
        Cm[r][c] = v;
        Cm[c][r] = v;
      }
    }
  } else if (!use_m) {
    for (int i = lane; i < m * m; i += kRRThreads) {
      const int r = i / m, c = i % m;
      Cm[r][c] = 0.5 * (G[r * ldg + c] + G[c * ldg + r]);
    }
  }
  __syncthreads();

  // ---- 2. FP32 Jacobi on fp32(C)
  for (int i = lane; i < mm * mm; i += kRRThreads) {
    const int r = i / mm, c = i % mm;
    A32[r][c] = (r < m && c < m) ? (float)Cm[r][c] : (r == c ? 1e30f : 0.0f);
    Q32[r][c] = (r == c) ? 1.0f : 0.0f;
  }
  __syncthreads();
  if (qkeep && warm && m >= 2) {
    // start from Q0 = diag(Q_old, 1): A = Q0^T C Q0 is diagonal but for its last row and
    // column (the leading block of C is the previous call's, as is the Cholesky factor's)
    const int mo = m - 1;
    for (int i = lane; i < mo * mo; i += kRRThreads)
      Q32[i / mo][i % mo] = (float)qkeep[(i / mo) * kMaxSub + i % mo];
    __syncthreads();
    for (int i = lane; i < m * m; i += kRRThreads) {  // T = A Q0
      const int r = i / m, c = i % m;
      float v = 0.0f;
      for (int k = 0; k < m; ++k) v = fmaf(A32[r][k], Q32[k][c], v);
      T32[r][c] = v;
    }
    __syncthreads();
    for (int i = lane; i < m * m; i += kRRThreads) {  // A = Q0^T T
      const int r = i / m, c = i % m;
      float v = 0.0f;
      for (int k = 0; k < m; ++k) v = fmaf(Q32[k][r], T32[k][c], v);
      A32[r][c] = v;
    }
    __syncthreads();
    for (int i = lane; i < m * m; i += kRRThreads) {  // symmetric part
      const int r = i / m, c = i % m;
      T32[r][c] = 0.5f * (A32[r][c] + A32[c][r]);
    }
    __syncthreads();
    for (int i = lane; i < m * m; i += kRRThreads) A32[i / m][i % m] = T32[i / m][i % m];
    __syncthreads();
  }
  jacobi_sweeps<float>(A32, Q32, m, mm, reinterpret_cast<float*>(cs64), pr,
                       reinterpret_cast<float (*)[2]>(red64));
  if (lane < m) lam[lane] = A32[lane][lane];
  __syncthreads();
  // lowest and second-lowest FP32 eigenvalues (lowest index on ties), spectral scale
  int c0 = 0;
  float l0 = lam[0], l1 = 3.0e38f, sc = fabsf(lam[0]);
  for (int j = 1; j < m; ++j) {
    const float v = lam[j];
    sc = fmaxf(sc, fabsf(v));
    if (v < l0) {
      l1 = l0;
      l0 = v;
      c0 = j;
    } else if (v < l1) {
      l1 = v;
    }
  }
  const double tol_r = 16.0 * (double)m * 1.1102230246251565e-16 * fmax((double)sc, 1e-300);

  // ---- 3. FP64 refinement of the lowest pair
  bool refined = false;
  if (m == 1 || (double)l1 - (double)l0 > 1e-5 * (double)sc) {
    if (w == 0) {
      double zi = l < m ? (double)Q32[l][c0] : 0.0;
      zi *= rsqrt64(warp_sum64(zi * zi));
      if (l < m) z[l] = zi;
    }
    __syncthreads();
    for (int it = 0; it <= 8; ++it) {
      if (l < m) {  // partial C z over the columns j = w, w + 4, ...
        double v = 0.0;
        for (int j = w; j < m; j += kRRThreads / 32) v = fma(Cm[l][j], z[j], v);
        part[w][l] = v;
      }
      __syncthreads();
      if (w == 0) {
        double czi = 0.0, zi = 0.0;
        if (l < m) {
          zi = z[l];
          for (int p = 0; p < kRRThreads / 32; ++p) czi += part[p][l];
        }
        const double th = warp_sum64(zi * czi);
        const double ri = czi - th * zi;
        float rr = (float)ri * (float)ri;  // the test needs no more than FP32
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rr += __shfl_xor_sync(full, rr, o);
        const bool done = (double)rr <= tol_r * tol_r;
        if (done || it == 8) {
          if (l == 0) {
            s_flag = done ? 1 : 2;
            s_theta = th;
          }
        } else {
          if (l < m) rbuf[l] = (float)ri;
          __syncwarp();
          if (l < m) {
            float pj = 0.0f;
            for (int i = 0; i < m; ++i) pj = fmaf(Q32[i][l], rbuf[i], pj);
            pbuf[l] = (l == c0) ? 0.0f : pj / (lam[l] - (float)th);
          }
          __syncwarp();
          float di = 0.0f;
          if (l < m)
            for (int j = 0; j < m; ++j) di = fmaf(Q32[l][j], pbuf[j], di);
          double zn = l < m ? zi - (double)di : 0.0;
          zn *= rsqrt64(warp_sum64(zn * zn));
          if (l < m) z[l] = zn;
          if (l == 0) s_flag = 0;
        }
      }
      __syncthreads();
      if (s_flag) break;
    }
    refined = s_flag == 1;
    __syncthreads();
  }

  // ---- 4. FP64 Jacobi on C when the FP32 solve is not enough
  double (*Q64)[kMaxSub + 1] = U;
  if (!refined) {
    for (int i = lane; i < mm * mm; i += kRRThreads) {
      const int r = i / mm, c = i % mm;
      X[r][c] = (r < m && c < m) ? Cm[r][c] : (r == c ? 1e300 : 0.0);
      Q64[r][c] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    jacobi_sweeps<double>(X, Q64, m, mm, cs64, pr, red64);
    if (lane == 0) {
      c0 = 0;
      for (int j = 1; j < m; ++j)
        if (X[j][j] < X[c0][c0]) c0 = j;
      s_theta = X[c0][c0];
    }
    __syncthreads();
    c0 = 0;
    for (int j = 1; j < m; ++j)
      if (X[j][j] < X[c0][c0]) c0 = j;
    if (w == 0) {  // the lowest eigenvector, normalised, into z
      double zi = l < m ? Q64[l][c0] : 0.0;
      zi *= rsqrt64(warp_sum64(zi * zi));
      if (l < m) z[l] = zi;
    }
  }
  __syncthreads();
  if (qkeep)
    for (int i = lane; i < m * m; i += kRRThreads)
      qkeep[(i / m) * kMaxSub + i % m] = refined ? (double)Q32[i / m][i % m] : Q64[i / m][i % m];

  // ---- 5. outputs: the lowest pair (y = L^-T z by columns of L in warp 0)
  const double theta = s_theta;
  if (w == 0) {
    double v = l < m ? z[l] : 0.0;
    if (use_m) {  // y = M z (M symmetric)
      v = 0.0;
      if (l < m)
        for (int j = 0; j < m; ++j) v = fma(L[l][j], z[j], v);
    } else if (use_s) {
      for (int i = m - 1; i >= 0; --i) {
        const double yi = __shfl_sync(full, v * Linv[l < m ? l : 0], i);
        if (l < i) v = fma(-L[i][l], yi, v);
        else if (l == i) v = yi;
      }
    }
    // sign: largest |component| positive (lowest index on ties)
    double big = l < m ? fabs(v) : -1.0;
    int arg = l;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double b2 = __shfl_xor_sync(full, big, o);
      const int a2 = __shfl_xor_sync(full, arg, o);
      if (b2 > big || (b2 == big && a2 < arg)) {
        big = b2;
        arg = a2;
      }
    }
    const double sv = __shfl_sync(full, v, arg);
    const double sg = sv < 0.0 ? -1.0 : 1.0;
    if (l == 0) {
      out[0] = theta;
      if (path) *path = (use_m ? 1 : 0) | (use_s ? 2 : 0) | (refined ? 4 : 0);
    }
    out[1 + l] = l < m ? sg * v : 0.0;
    if (all) {  // rank 0 of the ordered list: the same pair without the sign choice
      if (l == 0) all[0] = theta;
      all[1 + l] = l < m ? v : 0.0;
    }
  }
  if (!all) return;
  // ranks of the other eigenvalues (ascending, ties by index); rank 0 is c0
  if (lane < m) {
    const double lj = refined ? (double)lam[lane] : X[lane][lane];
    int r = 0;
    for (int k = 0; k < m; ++k) {
      const double lk = refined ? (double)lam[k] : X[k][k];
      if (lk < lj || (lk == lj && k < lane)) ++r;
    }
    rank_of[lane] = r;
  }
  __syncthreads();
  if (my_col < m && my_col != c0) {  // one thread per column, spread over the warps
    const int col = my_col;
    double zz[kMaxSub];
    double nz = 0.0;
    for (int r = 0; r < m; ++r) {
      zz[r] = refined ? (double)Q32[r][col] : Q64[r][col];
      nz = fma(zz[r], zz[r], nz);
    }
    nz = rsqrt64(nz);
    for (int r = 0; r < m; ++r) zz[r] *= nz;
    double* o = all + (size_t)rank_of[col] * kRitzStride;
    if (use_m) {  // y = M z
      for (int r = 0; r < m; ++r) {
        double v = 0.0;
        for (int k = 0; k < m; ++k) v = fma(L[r][k], zz[k], v);
        o[1 + r] = v;
      }
    } else {
      if (use_s) {  // y = L^-T z
        for (int i = m - 1; i >= 0; --i) {
          double v = zz[i];
          for (int k = i + 1; k < m; ++k) v -= L[k][i] * zz[k];
          zz[i] = v * Linv[i];
        }
      }
      for (int r = 0; r < m; ++r) o[1 + r] = zz[r];
    }
    o[0] = refined ? (double)lam[col] : X[col][col];
    for (int r = m; r < kMaxSub; ++r) o[1 + r] = 0.0;
  }
}

// argmin of D (lowest index on ties) -> idx[0], in two passes: the smallest value
// (mapped to an order-preserving uint64; min over a thread's elements, then the warp,
// then the block, one atomicMin per block), then the lowest index holding it
__global__ void k_argmin(const double* __restrict__ D, int64_t N, unsigned long long* best) {
  __shared__ unsigned long long wmin[32];
  unsigned long long m = ~0ull;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long u = (unsigned long long)__double_as_longlong(D[j]);
    u = (u >> 63) ? ~u : (u | 0x8000000000000000ull);
    m = u < m ? u : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v < m ? v : m;
  }
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = wmin[w] < m ? wmin[w] : m;
    atomicMin(best, m);
  }
}
__global__ void k_argmin_index(const double* __restrict__ D, int64_t N,
                               const unsigned long long* best, unsigned long long* idx) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long u = (unsigned long long)__double_as_longlong(D[j]);
    u = (u >> 63) ? ~u : (u | 0x8000000000000000ull);
    if (u == *best) atomicMin(idx, (unsigned long long)j);
  }
}
// The cold guess: the unit vector at the lowest diagonal entry plus a seeded
// perturbation of norm ~1e-3 (components eps * u_j, u_j uniform in [-1, 1) from
// SplitMix64 (Steele, Lea and Flood 2014) of the index j).  A unit vector alone has no
// component along eigenvectors that H never couples to it (the Krylov space of e_k
// misses them, e.g. a ground state of another spin than the lowest determinant), and
// Davidson would then converge to the lowest state it can reach instead of the lowest.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void k_unit(double* x, int64_t N, const unsigned long long* idx) {
  const double eps = 1e-3 * sqrt(3.0 / (double)N);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    const double u = (double)(splitmix64((uint64_t)j) >> 11) * 0x1.0p-52 - 1.0;
    x[j] = ((j == (int64_t)*idx) ? 1.0 : 0.0) + eps * u;
  }
}

__global__ void k_set_G(double* G, int ldg, int col, const double* vals, int m, int row_off) {
  int i = threadIdx.x;
  if (i < m) {
    G[(row_off + i) * ldg + col] = vals[i];
    G[col * ldg + row_off + i] = vals[i];
  }
}

__global__ void k_f64_to_f32(const double* __restrict__ x, float* __restrict__ y, int64_t N) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x)
    y[j] = (float)x[j];
}

// ------------------------------------------------------------ host helpers --

struct Ctx {
  const hinqs_ham_s* H;
  const hinqs_subspace_s* B;
  const hinqs_links_s* la;
  const hinqs_links_s* lb;
  cudaStream_t s;
  int64_t N;
  int grid;
  const hinqs_detlist_s* L = nullptr;  // basis list (vectors over its entries) or NULL
  SigmaBatcher* batcher = nullptr;     // lockstep batch this solve belongs to, or NULL
  cudaEvent_t ready = nullptr;         // this solve's event for the batcher
  double* partial = nullptr;  // [kPartial] >= kResGrid
  double* small = nullptr;    // scratch [4 * (kMaxSub+2)]
  float* t32 = nullptr;       // FP32 work vector [N] (mixed mode)
  unsigned int* counters = nullptr;  // [kMaxSub + 1] arrival counters of the dot kernels (zero)
};

// y = H x on the product subspace, or P H P x on the basis list when the context has one
static int apply_sigma(Ctx& c, const void* x, void* y, int precision) {
  if (c.L) return sigma_list_launch(c.H, c.B, c.la, c.lb, c.L, x, y, precision, c.s);
  if (c.batcher)
    return batcher_sigma(c.batcher, SigmaReq{c.H, c.B, c.la, c.lb, x, y, precision}, c.s, c.ready);
  return sigma_launch(c.H, c.B, c.la, c.lb, x, y, precision, c.s);
}

template <typename TA, typename TB>
static int dots(Ctx& c, const TA* A, int64_t lda, int m, const TB* b, double* out) {
  if (m <= 0) return HINQS_OK;
  k_dots<TA, TB><<<dim3(kRedGrid, m), kRedThreads, 0, c.s>>>(A, lda, b, c.N, c.partial,
                                                               c.counters, out);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

// out1[i] = A_i . b1, out2[i] = A_i . b2 with one pass over A
template <typename TA, typename TB>
static int dots2(Ctx& c, const TA* A, int64_t lda, int m, const TB* b1, const TB* b2,
                 double* out1, double* out2) {
  if (m <= 0) return HINQS_OK;
  k_dots2<TA, TB><<<dim3(kRedGrid, m), kRedThreads, 0, c.s>>>(A, lda, b1, b2, c.N, c.partial,
                                                                c.counters, out1, out2);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

template <typename TA>
static int lincomb(Ctx& c, double* out, const TA* A, int64_t lda, int m, const double* coef,
                   int mode) {
  if (m <= 0) return HINQS_OK;
  k_lincomb<TA><<<c.grid, 256, 0, c.s>>>(out, A, lda, m, coef, c.N, mode);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

// Orthonormalise t (FP64, modified in place) against m FP64 basis vectors V,
// classical Gram-Schmidt twice; store the normalised result into dst.
// Returns the norm ratio after/before.
static int orthonormalise(Ctx& c, double* t, const double* V, int64_t ld, int m, double* dst,
                          double* ratio) {
  double* coef = c.small;  // [kMaxSub]
  double* nrm = c.small + kMaxSub + 1;
  double hn[2];
  HQ_TRY(dots<double, double>(c, t, c.N, 1, t, nrm));
  HQ_CUDA(cudaMemcpyAsync(&hn[0], nrm, sizeof(double), cudaMemcpyDeviceToHost, c.s));
  for (int pass = 0; pass < 2 && m > 0; ++pass) {
    HQ_TRY(dots<double, double>(c, V, ld, m, t, coef));
    HQ_TRY(lincomb<double>(c, t, V, ld, m, coef, -1));
  }
  HQ_TRY(dots<double, double>(c, t, c.N, 1, t, nrm));
  HQ_CUDA(cudaMemcpyAsync(&hn[1], nrm, sizeof(double), cudaMemcpyDeviceToHost, c.s));
  HQ_CUDA(cudaStreamSynchronize(c.s));
  *ratio = (hn[0] > 0.0) ? std::sqrt(hn[1] / hn[0]) : 0.0;
  if (hn[1] <= 0.0) return HINQS_OK;
  k_scale_store<double, double><<<c.grid, 256, 0, c.s>>>(t, nrm, dst, c.N);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

// Mixed mode: remove the FP64 vector x from t in FP64 (twice), round t to FP32,
// remove the m FP32 basis vectors V in FP32 arithmetic (twice) and store the
// normalised FP32 result into dst.  The projected pencil carries the exact
// overlap of the stored vectors, so FP32 orthogonality suffices here.
static int orthonormalise_mixed(Ctx& c, double* t, const double* x, const float* V, int64_t ld,
                                int m, float* dst, double* ratio) {
  double* coef = c.small;
  double* coefx = c.small + kMaxSub;
  double* nrm = c.small + kMaxSub + 1;
  double hn[2];
  HQ_TRY(dots<double, double>(c, t, c.N, 1, t, nrm));
  HQ_CUDA(cudaMemcpyAsync(&hn[0], nrm, sizeof(double), cudaMemcpyDeviceToHost, c.s));
  for (int pass = 0; pass < 2; ++pass) {
    HQ_TRY(dots<double, double>(c, x, c.N, 1, t, coefx));
    HQ_TRY(lincomb<double>(c, t, x, c.N, 1, coefx, -1));
  }
  k_f64_to_f32<<<c.grid, 256, 0, c.s>>>(t, c.t32, c.N);
  for (int pass = 0; pass < 2 && m > 0; ++pass) {
    HQ_TRY(dots<float, float>(c, V, ld, m, c.t32, coef));
    k_lincomb_sub_f32<<<c.grid, 256, 0, c.s>>>(c.t32, V, ld, m, coef, c.N);
  }
  HQ_TRY(dots<float, float>(c, c.t32, c.N, 1, c.t32, nrm));
  HQ_CUDA(cudaMemcpyAsync(&hn[1], nrm, sizeof(double), cudaMemcpyDeviceToHost, c.s));
  HQ_CUDA(cudaStreamSynchronize(c.s));
  *ratio = (hn[0] > 0.0) ? std::sqrt(hn[1] / hn[0]) : 0.0;
  if (hn[1] <= 0.0) return HINQS_OK;
  k_scale_store<float, float><<<c.grid, 256, 0, c.s>>>(c.t32, nrm, dst, c.N);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

static int unit_at_min(Ctx& c, const double* D, double* x) {
  unsigned long long* b = reinterpret_cast<unsigned long long*>(c.small + 3 * kMaxSub);
  HQ_CUDA(cudaMemsetAsync(b, 0xff, 2 * sizeof(unsigned long long), c.s));
  k_argmin<<<c.grid, 256, 0, c.s>>>(D, c.N, b);
  k_argmin_index<<<c.grid, 256, 0, c.s>>>(D, c.N, b, b + 1);
  k_unit<<<c.grid, 256, 0, c.s>>>(x, c.N, b + 1);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

struct Trace {
  const hinqs_davidson_opts* o;
  int len = 0;
  std::chrono::steady_clock::time_point t0;
  void add(double theta, double resid, int kind) {
    if (!o || len >= o->trace_cap) return;
    double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (o->trace_theta) o->trace_theta[len] = theta;
    if (o->trace_resid) o->trace_resid[len] = resid;
    if (o->trace_time) o->trace_time[len] = t;
    if (o->trace_kind) o->trace_kind[len] = kind;
    ++len;
  }
};

// ---------------------------------------------------------------- FP64 ----

__global__ void k_init_pencil(double* G, double* S, const double* theta) {
  for (int i = threadIdx.x; i < kMaxSub * kMaxSub; i += blockDim.x) {
    G[i] = 0.0;
    if (S) S[i] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    G[0] = theta ? theta[0] : 0.0;
    if (S) S[0] = 1.0;
  }
}

// vectors kept at a restart: FP64 solver (current + previous + next Ritz vectors) and
// mixed solver (anchor + FP32 Ritz vectors); restart_keep = 0 takes the defaults
static int restart_keep_fp64(const hinqs_davidson_opts& o) {
  const int k = o.restart_keep > 0 ? o.restart_keep : kDefaultKeepFp64;
  return std::max(1, std::min(k, o.max_subspace - 1));
}
static int restart_keep_mixed(const hinqs_davidson_opts& o) {
  const int mmax = std::max(4, o.max_subspace);
  const int k = o.restart_keep > 0 ? o.restart_keep : kDefaultKeepMixed;
  return std::max(1, std::min(k, mmax - 2));
}

static int davidson_fp64(Ctx& c, const double* guess, const hinqs_davidson_opts& o, double* D,
                         double* energy, double* c_out, hinqs_davidson_info& info, Trace& tr) {
  const int mmax = o.max_subspace;
  const int kr = restart_keep_fp64(o);  // vectors kept at a restart
  const int64_t N = c.N;
  double *V = nullptr, *W = nullptr, *t = nullptr, *X = nullptr, *WX = nullptr, *G = nullptr,
         *ritz = nullptr, *col = nullptr, *ycoef = nullptr, *all = nullptr, *qk = nullptr;
  int rc = HINQS_OK;
  if ((rc = dalloc(&V, (size_t)mmax * N, c.s)) || (rc = dalloc(&W, (size_t)mmax * N, c.s)) ||
      (rc = dalloc(&t, N, c.s)) || (rc = dalloc(&X, (size_t)kr * N, c.s)) ||
      (rc = dalloc(&WX, (size_t)kr * N, c.s)) || (rc = dalloc(&G, kMaxSub * kMaxSub, c.s)) ||
      (rc = dalloc(&ritz, kMaxSub + 2, c.s)) || (rc = dalloc(&col, kMaxSub + 2, c.s)) ||
      (rc = dalloc(&ycoef, (size_t)kr * (kMaxSub + 2), c.s)) ||
      (rc = dalloc(&all, kMaxSub * kRitzStride, c.s)) ||
      (rc = dalloc(&qk, kMaxSub * kMaxSub, c.s))) {
  }
  auto cleanup = [&]() {
    dfree(qk, c.s);
    dfree(V, c.s);
    dfree(W, c.s);
    dfree(t, c.s);
    dfree(X, c.s);
    dfree(WX, c.s);
    dfree(G, c.s);
    dfree(ritz, c.s);
    dfree(col, c.s);
    dfree(ycoef, c.s);
    dfree(all, c.s);
  };
  if (rc) {
    cleanup();
    return rc;
  }
  auto run = [&]() -> int {
    if (guess) {
      HQ_CUDA(cudaMemcpyAsync(t, guess, N * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
    } else {
      HQ_TRY(unit_at_min(c, D, t));
    }
    double ratio;
    HQ_TRY(orthonormalise(c, t, V, N, 0, V, &ratio));
    if (ratio == 0.0) return fail(HINQS_ERR_ARG, "hinqs_davidson: zero initial guess");
    k_init_pencil<<<1, 256, 0, c.s>>>(G, nullptr, nullptr);
    int m = 1;
    double theta_prev = 0.0;
    bool have_prev = false;
    double hr[kMaxSub + 2] = {0}, hr_prev[kMaxSub + 2] = {0};
    int rr_warm = 0;  // the pencil grew by one column since the last k_rr
    for (int it = 0; it < o.max_iter; ++it) {
      double* vm = V + (size_t)(m - 1) * N;
      double* wm = W + (size_t)(m - 1) * N;
      HQ_TRY(apply_sigma(c, vm, wm, HINQS_PREC_FP64));
      info.n_sigma_fp64++;
      HQ_TRY(dots<double, double>(c, V, N, m, wm, col));
      k_set_G<<<1, kMaxSub, 0, c.s>>>(G, kMaxSub, m - 1, col, m, 0);
      k_rr<<<1, kRRThreads, 0, c.s>>>(G, kMaxSub, m, ritz, nullptr, nullptr, qk, rr_warm);
      rr_warm = 1;
      k_residual<double><<<kResGrid, kRedThreads, 0, c.s>>>(nullptr, nullptr, V, W, N, m, ritz, 0,
                                                            D, o.denom_floor, N, t, c.partial,
                                                            c.counters + kMaxSub, col + kMaxSub);
      HQ_LAUNCH_CHECK();
      double hres = 0.0;
      HQ_CUDA(cudaMemcpyAsync(hr, ritz, (kMaxSub + 1) * sizeof(double), cudaMemcpyDeviceToHost, c.s));
      HQ_CUDA(cudaMemcpyAsync(&hres, col + kMaxSub, sizeof(double), cudaMemcpyDeviceToHost, c.s));
      HQ_CUDA(cudaStreamSynchronize(c.s));
      double theta = hr[0], res = std::sqrt(std::max(hres, 0.0));
      info.iterations = it + 1;
      info.energy = theta;
      info.residual = res;
      tr.add(theta, res, 0);
      bool conv = res <= o.tol_residual && have_prev && std::fabs(theta - theta_prev) <= o.tol_energy;
      if (res <= o.tol_residual * 1e-3) conv = true;
      if (conv || it + 1 == o.max_iter) {
        HQ_TRY(lincomb<double>(c, c_out, V, N, m, ritz + 1, 0));
        info.status = conv ? HINQS_OK : HINQS_NOT_CONVERGED;
        if (energy) *energy = theta;
        return info.status;
      }
      theta_prev = theta;
      have_prev = true;
      if (m == mmax) {
        // Thick restart: keep the current Ritz vector, the previous one (the search
        // direction of the last step) and the next-lowest Ritz vectors, kr in all,
        // orthonormalised in the m-dimensional coefficient space (near convergence the
        // current and previous vectors are nearly parallel; doing this on the N-vectors
        // would lose orthogonality).  The kept pencil is Y G Y^T, formed on the host.
        k_rr<<<1, kRRThreads, 0, c.s>>>(G, kMaxSub, m, ritz, nullptr, all);
        HQ_LAUNCH_CHECK();
        std::vector<double> hall((size_t)kMaxSub * kRitzStride), hG((size_t)kMaxSub * kMaxSub);
        HQ_CUDA(cudaMemcpyAsync(hall.data(), all, hall.size() * sizeof(double),
                                cudaMemcpyDeviceToHost, c.s));
        HQ_CUDA(cudaMemcpyAsync(hG.data(), G, hG.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                c.s));
        HQ_CUDA(cudaStreamSynchronize(c.s));
        std::vector<std::vector<double>> Y;
        auto add = [&](std::vector<double> v) {
          for (int pass = 0; pass < 2; ++pass)
            for (const auto& u : Y) {
              double d = 0.0;
              for (int i = 0; i < m; ++i) d += u[i] * v[i];
              for (int i = 0; i < m; ++i) v[i] -= d * u[i];
            }
          double nn = 0.0;
          for (int i = 0; i < m; ++i) nn += v[i] * v[i];
          if (nn > 1e-24) {
            for (int i = 0; i < m; ++i) v[i] /= std::sqrt(nn);
            Y.push_back(v);
          }
        };
        std::vector<double> v(m);
        for (int i = 0; i < m; ++i) v[i] = hr[1 + i];
        add(v);
        if (kr >= 2) {
          for (int i = 0; i < m; ++i) v[i] = (i < m - 1) ? hr_prev[1 + i] : 0.0;
          add(v);
        }
        for (int j = 1; j < m && (int)Y.size() < kr; ++j) {
          for (int i = 0; i < m; ++i) v[i] = hall[(size_t)j * kRitzStride + 1 + i];
          add(v);
        }
        const int mnew = (int)Y.size();
        std::vector<double> hc((size_t)mnew * (kMaxSub + 2), 0.0);
        for (int j = 0; j < mnew; ++j)
          for (int i = 0; i < m; ++i) hc[(size_t)j * (kMaxSub + 2) + i] = Y[j][i];
        std::vector<double> hGn((size_t)kMaxSub * kMaxSub, 0.0);  // Y G Y^T
        for (int a2 = 0; a2 < mnew; ++a2)
          for (int b2 = 0; b2 < mnew; ++b2) {
            double acc = 0.0;
            for (int i = 0; i < m; ++i) {
              double gi = 0.0;
              for (int j = 0; j < m; ++j)
                gi += 0.5 * (hG[(size_t)i * kMaxSub + j] + hG[(size_t)j * kMaxSub + i]) * Y[b2][j];
              acc += Y[a2][i] * gi;
            }
            hGn[(size_t)a2 * kMaxSub + b2] = acc;
          }
        HQ_CUDA(cudaMemcpyAsync(ycoef, hc.data(), hc.size() * sizeof(double),
                                cudaMemcpyHostToDevice, c.s));
        for (int j = 0; j < mnew; ++j) {
          HQ_TRY(lincomb<double>(c, X + (size_t)j * N, V, N, m, ycoef + (size_t)j * (kMaxSub + 2), 0));
          HQ_TRY(lincomb<double>(c, WX + (size_t)j * N, W, N, m, ycoef + (size_t)j * (kMaxSub + 2), 0));
        }
        HQ_CUDA(cudaMemcpyAsync(V, X, (size_t)mnew * N * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
        HQ_CUDA(cudaMemcpyAsync(W, WX, (size_t)mnew * N * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
        HQ_CUDA(cudaMemcpyAsync(G, hGn.data(), hGn.size() * sizeof(double), cudaMemcpyHostToDevice,
                                c.s));
        // the current Ritz vector is now V[0]: its coefficients in the new basis
        for (int i = 1; i <= kMaxSub; ++i) hr[i] = (i == 1) ? 1.0 : 0.0;
        HQ_CUDA(cudaMemcpyAsync(ritz, hr, (kMaxSub + 1) * sizeof(double), cudaMemcpyHostToDevice,
                                c.s));
        HQ_CUDA(cudaStreamSynchronize(c.s));  // the host arrays above go out of scope
        m = mnew;
        rr_warm = 0;
        // the residual t of the current Ritz vector (now V[0]) is still valid
        info.n_restarts++;
      }
      std::copy(hr, hr + kMaxSub + 1, hr_prev);
      if (m < mmax) {
        HQ_TRY(orthonormalise(c, t, V, N, m, V + (size_t)m * N, &ratio));
        if (ratio < 1e-10) {
          // stagnated preconditioner: fall back to the plain residual direction
          k_residual<double><<<kResGrid, kRedThreads, 0, c.s>>>(nullptr, nullptr, V, W, N, m, ritz,
                                                                0, D, 1e300, N, t, c.partial);
          HQ_TRY(orthonormalise(c, t, V, N, m, V + (size_t)m * N, &ratio));
          if (ratio < 1e-14) {
            HQ_TRY(lincomb<double>(c, c_out, V, N, m, ritz + 1, 0));
            if (energy) *energy = info.energy;
            info.status = HINQS_NOT_CONVERGED;
            return info.status;
          }
        }
        m++;
      }
    }
    return HINQS_NOT_CONVERGED;
  };
  rc = run();
  cleanup();
  return rc;
}

// --------------------------------------------------------------- mixed ----
//
// Basis {x, v_1..v_m}: x is an FP64 unit vector (the anchor) with an FP64 product
// s = H x, the v_i are FP32 with FP32 products w_i.  The projected pencil (G, S) is
// FP64 with G_00 = x.s, G_0i = s.v_i, G_ij = v_i.w_j, S_0i = x.v_i, S_ij = v_i.v_j.
// Inner iterations add preconditioned residual directions (FP32 products).  A
// restart keeps the anchor's Ritz vector and the next keep-1 Ritz vectors (as FP32
// vectors with FP32-combined products).  The anchor's product after a restart is
// y_0 s + sum y_i w_i; an FP64 product replaces it (a refinement) when the inner
// residual falls below inner_tol times the last FP64 residual, or after
// kSoftRestarts restarts without one.  Convergence is judged on FP64 residuals.

constexpr int kSoftRestarts = 3;

// basis-vector bound of the fused passes for m vectors
static int vec_bound(int m) { return m <= 4 ? 4 : m <= 8 ? 8 : m <= 16 ? 16 : 32; }

// grid: one full wave, but no more blocks than 256-element chunks of the vectors (so
// that the passes of small problems leave the GPU to other streams' work)
template <template <int> class F, typename... A>
static void launch_mb(int m, int64_t n_elems, cudaStream_t s, A... a) {
  const int cap = (int)std::min<int64_t>(kVecGrid, std::max<int64_t>(1, (n_elems + 255) / 256));
  switch (vec_bound(m)) {
    case 4: F<4>::go(s, cap, a...); break;
    case 8: F<8>::go(s, cap, a...); break;
    case 16: F<16>::go(s, cap, a...); break;
    default: F<32>::go(s, cap, a...); break;
  }
}
// One full wave of a fused pass: the SMs times the blocks of the kernel that fit on
// one (its registers decide), at most kVecGrid (the partial-sum buffer).
template <typename K>
static int vec_grid(K kern) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRedThreads, 0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return std::min(kVecGrid, per_sm * kNumSMs);
}
template <int MB>
struct Res32 {
  template <typename... A>
  static void go(cudaStream_t s, int cap, A... a) {
    static const int g = vec_grid(k_res32<MB>);
    k_res32<MB><<<std::min(g, cap), kRedThreads, 0, s>>>(a...);
  }
};
template <int MB>
struct Ortho32 {
  template <typename... A>
  static void go(cudaStream_t s, int cap, A... a) {
    static const int g = vec_grid(k_ortho32<MB>);
    k_ortho32<MB><<<std::min(g, cap), kRedThreads, 0, s>>>(a...);
  }
};
template <int MB>
struct Col32 {
  template <typename... A>
  static void go(cudaStream_t s, int cap, A... a) {
    static const int g = vec_grid(k_col32<MB>);
    k_col32<MB><<<std::min(g, cap), kRedThreads, 0, s>>>(a...);
  }
};
template <int MB>
struct Restart32 {
  template <typename... A>
  static void go(cudaStream_t s, int cap, A... a) {
    static const int g = vec_grid(k_restart32<MB>);
    k_restart32<MB><<<std::min(g, cap), kRedThreads, 0, s>>>(a...);
  }
};
template <int MB>
struct Row32 {
  template <typename... A>
  static void go(cudaStream_t s, int cap, A... a) {
    static const int g = vec_grid(k_anchor_row32<MB>);
    k_anchor_row32<MB><<<std::min(g, cap), kRedThreads, 0, s>>>(a...);
  }
};

static int davidson_mixed(Ctx& c, const double* guess, const hinqs_davidson_opts& o, double* D,
                          double* energy, double* c_out, hinqs_davidson_info& info, Trace& tr) {
  const int mmax = std::max(4, o.max_subspace);  // pencil order 1 + m <= mmax
  const int keep = restart_keep_mixed(o);         // Ritz vectors kept at a restart (with x)
  const int64_t N = c.N;
  double *x = nullptr, *sx = nullptr, *t = nullptr, *xn = nullptr, *sxn = nullptr, *G = nullptr,
         *S = nullptr, *G1 = nullptr, *ritz = nullptr, *ritz1 = nullptr, *all = nullptr,
         *col = nullptr, *scol = nullptr, *vsum = nullptr, *qk = nullptr;
  float *V = nullptr, *W = nullptr, *U = nullptr, *WU = nullptr, *x32 = nullptr, *ra = nullptr,
        *D32 = nullptr;
  int rc = HINQS_OK;
  if ((rc = dalloc(&x, N, c.s)) || (rc = dalloc(&sx, N, c.s)) || (rc = dalloc(&t, N, c.s)) ||
      (rc = dalloc(&xn, N, c.s)) || (rc = dalloc(&sxn, N, c.s)) ||
      (rc = dalloc(&V, (size_t)mmax * N, c.s)) || (rc = dalloc(&W, (size_t)mmax * N, c.s)) ||
      (rc = dalloc(&U, (size_t)keep * N, c.s)) || (rc = dalloc(&WU, (size_t)keep * N, c.s)) ||
      (rc = dalloc(&G, kMaxSub * kMaxSub, c.s)) || (rc = dalloc(&S, kMaxSub * kMaxSub, c.s)) ||
      (rc = dalloc(&G1, kMaxSub * kMaxSub, c.s)) || (rc = dalloc(&ritz, kMaxSub + 2, c.s)) ||
      (rc = dalloc(&ritz1, kMaxSub + 2, c.s)) || (rc = dalloc(&all, kMaxSub * kRitzStride, c.s)) ||
      (rc = dalloc(&col, kMaxSub + 2, c.s)) || (rc = dalloc(&scol, kMaxSub + 2, c.s)) ||
      (rc = dalloc(&vsum, kVecOut, c.s)) || (rc = dalloc(&qk, kMaxSub * kMaxSub, c.s)) ||
      (rc = dalloc(&c.t32, N, c.s)) ||
      (rc = dalloc(&x32, N, c.s)) || (rc = dalloc(&ra, N, c.s)) || (rc = dalloc(&D32, N, c.s))) {
  }
  auto cleanup = [&]() {
    for (double* p : {x, sx, t, xn, sxn, G, S, G1, ritz, ritz1, all, col, scol, vsum, qk}) {
      double* q = p;
      dfree(q, c.s);
    }
    for (float* p : {V, W, U, WU, c.t32, x32, ra, D32}) {
      float* q = p;
      dfree(q, c.s);
    }
  };
  if (rc) {
    cleanup();
    return rc;
  }
  double* theta_a = c.small + 2 * kMaxSub + 2;  // x.s / x.x of the current anchor
  double* gs = c.small + 2 * kMaxSub + 6;       // {x.s, x.x}
  unsigned int* ctr = c.counters + kMaxSub;
  const float floor32 = (float)o.denom_floor;
  // the pencil column of V_j (pencil index j + 1) and its product W_j
  auto add_column = [&](int j) -> int {
    launch_mb<Col32>(j + 1, N, c.s, (const float*)x32, (const float*)ra, (const float*)V,
                     (const float*)W, (int64_t)N, j, N, c.partial, ctr, vsum);
    k_set_col32<<<1, kMaxSub + 1, 0, c.s>>>(G, S, kMaxSub, j + 1, vsum, j + 1, theta_a);
    HQ_LAUNCH_CHECK();
    return HINQS_OK;
  };
  auto run = [&]() -> int {
    k_f64_to_f32<<<c.grid, 256, 0, c.s>>>(D, D32, N);
    if (guess) {
      HQ_CUDA(cudaMemcpyAsync(t, guess, N * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
    } else {
      HQ_TRY(unit_at_min(c, D, t));
    }
    double ratio;
    HQ_TRY(orthonormalise(c, t, nullptr, N, 0, x, &ratio));
    if (ratio == 0.0) return fail(HINQS_ERR_ARG, "hinqs_davidson: zero initial guess");
    k_init_pencil<<<1, 256, 0, c.s>>>(G, S, nullptr);
    int m = 0, soft = 0, total = 0;
    bool hard = true, have_prev = false;
    double theta_prev = 0.0, target = 0.0;
    double h[2];
    std::vector<double> hs(kVecOut + 1);
    for (;;) {
      if (hard) {
        HQ_TRY(apply_sigma(c, x, sx, o.refine_precision));
        info.n_sigma_fp64++;
        total++;
        double* th = c.small + 2 * kMaxSub;
        HQ_TRY(dots<double, double>(c, x, N, 1, sx, th));
        k_init_pencil<<<1, 256, 0, c.s>>>(G1, nullptr, th);
        k_rr<<<1, kRRThreads, 0, c.s>>>(G1, kMaxSub, 1, ritz1, nullptr);  // (theta, 1)
        k_residual<float><<<kResGrid, kRedThreads, 0, c.s>>>(x, sx, V, W, N, 0, ritz1, 1, D,
                                                             o.denom_floor, N, t, c.partial,
                                                             c.counters + kMaxSub, col + kMaxSub);
        HQ_LAUNCH_CHECK();
        HQ_CUDA(cudaMemcpyAsync(&h[0], ritz1, sizeof(double), cudaMemcpyDeviceToHost, c.s));
        HQ_CUDA(cudaMemcpyAsync(&h[1], col + kMaxSub, sizeof(double), cudaMemcpyDeviceToHost, c.s));
        HQ_CUDA(cudaStreamSynchronize(c.s));
        const double theta = h[0], res = std::sqrt(std::max(h[1], 0.0));
        info.energy = theta;
        info.residual = res;
        info.iterations++;
        tr.add(theta, res, 0);
        bool conv = res <= o.tol_residual && have_prev && std::fabs(theta - theta_prev) <= o.tol_energy;
        if (res <= o.tol_residual * 1e-3) conv = true;
        if (conv || total >= o.max_iter) {
          HQ_CUDA(cudaMemcpyAsync(c_out, x, N * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
          if (energy) *energy = theta;
          info.status = conv ? HINQS_OK : HINQS_NOT_CONVERGED;
          return info.status;
        }
        theta_prev = theta;
        have_prev = true;
        info.n_refinements++;
        target = std::max(o.inner_tol * res, 0.3 * o.tol_residual);
        soft = 0;
        hard = false;
      }
      // the anchor in FP32 form and row / column 0 of the pencil
      HQ_TRY(dots2<double, double>(c, x, N, 1, sx, x, gs, gs + 1));
      k_anchor32<<<c.grid, 256, 0, c.s>>>(x, sx, gs, theta_a, x32, ra, N);
      k_set_G<<<1, kMaxSub, 0, c.s>>>(G, kMaxSub, 0, gs, 1, 0);
      k_set_G<<<1, kMaxSub, 0, c.s>>>(S, kMaxSub, 0, gs + 1, 1, 0);
      if (m > 0) {
        launch_mb<Row32>(m, N, c.s, (const float*)x32, (const float*)ra, (const float*)V, (int64_t)N,
                         m, N, c.partial, ctr, vsum);
        k_set_row32<<<1, kMaxSub, 0, c.s>>>(G, S, kMaxSub, vsum, m, theta_a);
      }
      HQ_LAUNCH_CHECK();
      if (m == 0) {  // first direction: the preconditioned FP64 residual in t
        HQ_TRY(orthonormalise_mixed(c, t, x, V, N, 0, V, &ratio));
        HQ_TRY(apply_sigma(c, V, W, o.inner_precision));
        info.n_sigma_fp32++;
        total++;
        m = 1;
        HQ_TRY(add_column(0));
      }
      bool restart_hard = false;
      int rr_warm = 0;  // the pencil grew by one column since the last k_rr
      for (;;) {
        // residual and correction of the pencil's lowest Ritz pair, with the dot products
        // of its Gram-Schmidt pass against {x, V}
        k_rr<<<1, kRRThreads, 0, c.s>>>(G, kMaxSub, m + 1, ritz, S, nullptr, qk, rr_warm);
        rr_warm = 1;
        launch_mb<Res32>(m, N, c.s, (const float*)ra, (const float*)x32, (const float*)V,
                         (const float*)W, (int64_t)N, m, (const double*)ritz, (const double*)theta_a,
                         (const float*)D32, floor32, N, c.t32, c.partial, ctr, vsum);
        HQ_LAUNCH_CHECK();
        HQ_CUDA(cudaMemcpyAsync(hs.data(), ritz, sizeof(double), cudaMemcpyDeviceToHost, c.s));
        HQ_CUDA(cudaMemcpyAsync(hs.data() + 1, vsum, (m + 3) * sizeof(double),
                                cudaMemcpyDeviceToHost, c.s));
        HQ_CUDA(cudaStreamSynchronize(c.s));
        const double rin = std::sqrt(std::max(hs[1], 0.0));
        info.iterations++;
        tr.add(hs[0], rin, 1);
        if (rin <= target || total >= o.max_iter) {
          restart_hard = true;
          break;
        }
        if (m + 1 >= mmax) {
          restart_hard = (++soft > kSoftRestarts);
          break;
        }
        // classical Gram-Schmidt against {x, V} (unit vectors up to FP32 rounding; the
        // pencil carries their exact overlaps): one pass when it keeps more than half
        // of |t|^2 (then a second pass would change nothing that matters), else a
        // second pass from the dot products of the first
        const double tt = hs[2];
        OrthoCoef cf;
        double p2 = tt;
        cf.c[0] = (float)hs[3];
        p2 -= hs[3] * hs[3];
        for (int i = 0; i < m; ++i) {
          cf.c[1 + i] = (float)hs[4 + i];
          p2 -= hs[4 + i] * hs[4 + i];
        }
        float* vm = V + (size_t)m * N;
        if (!(tt > 0.0)) {
          restart_hard = true;
          break;
        }
        if (p2 > 0.5 * tt) {
          cf.scale = (float)(1.0 / std::sqrt(p2));
          launch_mb<Ortho32>(m, N, c.s, (const float*)c.t32, (const float*)x32, (const float*)V,
                             (int64_t)N, m, cf, vm, N, c.partial, ctr, vsum);
        } else {
          cf.scale = 1.0f;
          launch_mb<Ortho32>(m, N, c.s, (const float*)c.t32, (const float*)x32, (const float*)V,
                             (int64_t)N, m, cf, vm, N, c.partial, ctr, vsum);
          HQ_CUDA(cudaMemcpyAsync(hs.data(), vsum, (m + 2) * sizeof(double), cudaMemcpyDeviceToHost,
                                  c.s));
          HQ_CUDA(cudaStreamSynchronize(c.s));
          const double oo = hs[m + 1];
          if (!(oo > 1e-24 * tt)) {  // t lies in span{x, V}: no new direction
            restart_hard = true;
            break;
          }
          double q2 = oo;
          for (int i = 0; i <= m; ++i) {
            cf.c[i] = (float)hs[i];
            q2 -= hs[i] * hs[i];
          }
          cf.scale = (float)(1.0 / std::sqrt(q2 > 0.5 * oo ? q2 : oo));
          launch_mb<Ortho32>(m, N, c.s, (const float*)vm, (const float*)x32, (const float*)V,
                             (int64_t)N, m, cf, vm, N, c.partial, ctr, vsum);
        }
        HQ_LAUNCH_CHECK();
        HQ_TRY(apply_sigma(c, vm, W + (size_t)m * N, o.inner_precision));
        info.n_sigma_fp32++;
        total++;
        HQ_TRY(add_column(m));
        m++;
      }
      // restart: anchor = lowest Ritz vector, plus keep-1 FP32 Ritz vectors (every
      // eigenpair of the final pencil, solved again: the iterations ask for the lowest only)
      const int kk = std::min(keep, m + 1);
      k_rr<<<1, kRRThreads, 0, c.s>>>(G, kMaxSub, m + 1, ritz, S, all);
      // xn = y0 x + V y, sxn = y0 s + W y (FP64) and the kept FP32 Ritz vectors with their
      // products, in one pass (the FP32 parts carry the correction)
      launch_mb<Restart32>(std::max(m, 1), N, c.s, (const double*)x, (const double*)sx,
                           (const float*)x32, (const float*)ra, (const float*)V, (const float*)W,
                           (int64_t)N, m, (const double*)all, kk, (const double*)theta_a, N, xn,
                           sxn, U, WU);
      HQ_LAUNCH_CHECK();
      // normalise the anchor (y^T S y = 1 up to rounding) and its product alike
      double* nrm = c.small + 2 * kMaxSub + 1;
      HQ_TRY(dots<double, double>(c, xn, N, 1, xn, nrm));
      k_scale_store<double, double><<<c.grid, 256, 0, c.s>>>(xn, nrm, x, N);
      k_scale_store<double, double><<<c.grid, 256, 0, c.s>>>(sxn, nrm, sx, N);
      m = kk - 1;
      if (m > 0) {
        HQ_CUDA(cudaMemcpyAsync(V, U, (size_t)m * N * sizeof(float), cudaMemcpyDeviceToDevice, c.s));
        HQ_CUDA(cudaMemcpyAsync(W, WU, (size_t)m * N * sizeof(float), cudaMemcpyDeviceToDevice, c.s));
      }
      k_init_pencil<<<1, 256, 0, c.s>>>(G, S, nullptr);
      HQ_LAUNCH_CHECK();
      for (int j = 1; j <= m; ++j) {
        const float* v = V + (size_t)(j - 1) * N;
        const float* w = W + (size_t)(j - 1) * N;
        HQ_TRY(dots2<float, float>(c, V, N, j, w, v, col + 1, scol + 1));
        k_set_G<<<1, kMaxSub, 0, c.s>>>(G, kMaxSub, j, col + 1, j, 1);
        k_set_G<<<1, kMaxSub, 0, c.s>>>(S, kMaxSub, j, scol + 1, j, 1);
      }
      HQ_LAUNCH_CHECK();
      info.n_restarts++;
      hard = restart_hard;
    }
  };
  rc = run();
  cleanup();
  return rc;
}

}  // namespace hinqs

using namespace hinqs;

extern "C" void hinqs_davidson_default_opts(hinqs_davidson_opts* o) {
  if (!o) return;
  o->precision = HINQS_DAVIDSON_FP64;
  o->max_iter = 200;
  o->max_subspace = 16;
  o->tol_residual = 1e-8;
  o->tol_energy = 1e-10;
  o->denom_floor = 1e-4;
  o->inner_tol = 1e-3;
  o->trace_cap = 0;
  o->trace_theta = nullptr;
  o->trace_resid = nullptr;
  o->trace_time = nullptr;
  o->trace_kind = nullptr;
  o->inner_precision = HINQS_PREC_FP32;
  o->restart_keep = 0;
  o->refine_precision = HINQS_PREC_FP64_DFAB;
}

// Device bytes one hinqs_davidson call requests from the stream-ordered pool at its
// peak: the context (partials, scratch, counters, the diagonal), the solver's vectors
// and pencils (as allocated by davidson_fp64 / davidson_mixed above) and the two
// N-element temporaries of an FP64 sigma product.  Keep in step with those allocations.
static size_t davidson_workspace_bytes(int64_t N, const hinqs_davidson_opts& o) {
  const size_t d = sizeof(double), f = sizeof(float);
  size_t b = ((size_t)kPartial + 4 * (kMaxSub + 2)) * d +
             (kMaxSub + 1) * sizeof(unsigned int) + (size_t)N * d;
  if (o.precision == HINQS_DAVIDSON_FP64) {
    const size_t mmax = (size_t)o.max_subspace, kr = (size_t)restart_keep_fp64(o);
    b += (2 * mmax + 1 + 2 * kr) * (size_t)N * d;               // V, W, t, X[kr], WX[kr]
    b += (2 * (size_t)kMaxSub * kMaxSub + (2 + kr) * (kMaxSub + 2) + (size_t)kMaxSub * kRitzStride) * d;
  } else {
    const size_t mmax = (size_t)std::max(4, o.max_subspace);
    const size_t keep = (size_t)restart_keep_mixed(o);
    b += 5 * (size_t)N * d;                                     // x, sx, t, xn, sxn
    b += (2 * mmax + 2 * keep + 4) * (size_t)N * f;             // V, W, U, WU, t32, x32, ra, D32
    b += (4 * (size_t)kMaxSub * kMaxSub + 4 * (kMaxSub + 2) + (size_t)kMaxSub * kRitzStride +
          kVecOut) * d;
  }
  // sigma temporaries of the FP64 (or double-float) product
  const bool df = o.precision == HINQS_DAVIDSON_MIXED && o.refine_precision == HINQS_PREC_FP64_DFAB;
  return b + (df ? 3 : 2) * (size_t)N * d;
}

extern "C" int hinqs_davidson_workspace_size(int64_t n_alpha_strings, int64_t n_beta_strings,
                                             const hinqs_davidson_opts* opts, size_t* bytes) {
  if (!bytes || n_alpha_strings < 0 || n_beta_strings < 0)
    return fail(HINQS_ERR_ARG, "hinqs_davidson_workspace_size: NULL output or negative size");
  hinqs_davidson_opts o;
  hinqs_davidson_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_subspace < 3 || o.max_subspace > kMaxSub)
    return fail(HINQS_ERR_ARG, "hinqs_davidson_workspace_size: max_subspace must be in 3..%d",
                kMaxSub);
  if (o.precision != HINQS_DAVIDSON_FP64 && o.precision != HINQS_DAVIDSON_MIXED)
    return fail(HINQS_ERR_ARG, "hinqs_davidson_workspace_size: unknown precision %d", o.precision);
  *bytes = davidson_workspace_bytes(n_alpha_strings * n_beta_strings, o);
  return HINQS_OK;
}

int hinqs::davidson_run(const hinqs_ham* H, const hinqs_subspace* B, const hinqs_links* la,
                        const hinqs_links* lb, const hinqs_detlist* L, const double* guess,
                        const hinqs_davidson_opts* opts, double* energy, double* c_out,
                        hinqs_davidson_info* info_out, void* stream, const char* who,
                        SigmaBatcher* batcher, cudaEvent_t ready) {
  HQ_TRY(check_triplet(H, B, la, lb, who));
  if (L) {
    HQ_TRY(check_list(B, L, who));
    if (L->m == 0) return fail(HINQS_ERR_EMPTY, "%s: empty basis list", who);
  }
  if (!c_out) return fail(HINQS_ERR_ARG, "%s: c_out is NULL", who);
  hinqs_davidson_opts o;
  hinqs_davidson_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_subspace < 3 || o.max_subspace > kMaxSub)
    return fail(HINQS_ERR_ARG, "%s: max_subspace must be in 3..%d", who, kMaxSub);
  if (o.max_iter < 1 || !(o.tol_residual > 0.0) || !(o.denom_floor > 0.0))
    return fail(HINQS_ERR_ARG, "%s: bad max_iter / tolerances", who);
  if (o.precision != HINQS_DAVIDSON_FP64 && o.precision != HINQS_DAVIDSON_MIXED)
    return fail(HINQS_ERR_ARG, "%s: unknown precision %d", who, o.precision);
  if (o.precision == HINQS_DAVIDSON_MIXED && o.inner_precision != HINQS_PREC_FP32 &&
      o.inner_precision != HINQS_PREC_FP32_BF16AB && o.inner_precision != HINQS_PREC_FP32_BF16X3AB &&
      o.inner_precision != HINQS_PREC_FP32_BF16C)
    return fail(HINQS_ERR_ARG, "%s: unknown inner precision %d", who, o.inner_precision);
  if (o.precision == HINQS_DAVIDSON_MIXED && o.refine_precision != HINQS_PREC_FP64 &&
      o.refine_precision != HINQS_PREC_FP64_DFAB)
    return fail(HINQS_ERR_ARG, "%s: unknown refinement precision %d", who, o.refine_precision);
  // the list operator has no tensor-core form: its inner products run in FP32
  if (L && o.precision == HINQS_DAVIDSON_MIXED) o.inner_precision = HINQS_PREC_FP32;
  hinqs_davidson_info info{};
  Trace tr;
  tr.o = &o;
  tr.t0 = std::chrono::steady_clock::now();
  Ctx c{H, B, la, lb, (cudaStream_t)stream, L ? L->m : B->Na * B->Nb, 0};
  c.L = L;
  if (!L) {
    c.batcher = batcher;
    c.ready = ready;
  }
  c.grid = (int)std::min<int64_t>(ceil_div(c.N, 256), 8 * kNumSMs);
  double* D = nullptr;
  int rc = HINQS_OK;
  if ((rc = dalloc(&c.partial, kPartial, c.s)) ||
      (rc = dalloc(&c.small, 4 * (kMaxSub + 2), c.s)) ||
      (rc = dalloc(&c.counters, kMaxSub + 1, c.s)) || (rc = dalloc(&D, c.N, c.s))) {
  }
  if (!rc && cudaMemsetAsync(c.counters, 0, (kMaxSub + 1) * sizeof(unsigned int), c.s) != cudaSuccess)
    rc = cuda_fail(cudaGetLastError(), "hinqs_davidson counters", __FILE__, __LINE__);
  if (!rc) rc = L ? diag_list_launch(H, la, lb, L, D, c.s) : diag_launch(H, B, la, lb, D, c.s);
  if (!rc) {
    if (o.precision == HINQS_DAVIDSON_FP64)
      rc = davidson_fp64(c, guess, o, D, energy, c_out, info, tr);
    else
      rc = davidson_mixed(c, guess, o, D, energy, c_out, info, tr);
  }
  if (rc >= 0) {
    cudaError_t e = cudaStreamSynchronize(c.s);
    if (e != cudaSuccess) rc = cuda_fail(e, who, __FILE__, __LINE__);
  }
  if (rc >= 0 && o.precision == HINQS_DAVIDSON_MIXED && o.inner_precision != HINQS_PREC_FP32) {
    int t = tc_error_check(c.s);
    if (t < 0) rc = t;
  }
  dfree(c.partial, c.s);
  dfree(c.small, c.s);
  dfree(c.counters, c.s);
  dfree(D, c.s);
  info.trace_len = tr.len;
  info.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - tr.t0).count();
  if (rc >= 0) info.status = rc;
  if (info_out) *info_out = info;
  return rc;
}

extern "C" int hinqs_davidson(const hinqs_ham* H, const hinqs_subspace* B, const hinqs_links* la,
                              const hinqs_links* lb, const double* guess,
                              const hinqs_davidson_opts* opts, double* energy, double* c_out,
                              hinqs_davidson_info* info_out, void* stream) {
  return davidson_run(H, B, la, lb, nullptr, guess, opts, energy, c_out, info_out, stream,
                      "hinqs_davidson", nullptr, nullptr);
}

extern "C" int hinqs_davidson_list(const hinqs_ham* H, const hinqs_subspace* B,
                                   const hinqs_links* la, const hinqs_links* lb,
                                   const hinqs_detlist* L, const double* guess,
                                   const hinqs_davidson_opts* opts, double* energy, double* c_out,
                                   hinqs_davidson_info* info_out, void* stream) {
  return davidson_run(H, B, la, lb, L, guess, opts, energy, c_out, info_out, stream,
                      "hinqs_davidson_list", nullptr, nullptr);
}

extern "C" int hinqs_selftest_projected_eig(const double* G, const double* S, int m,
                                            double* theta_y, double* pairs, int* path,
                                            void* stream) {
  using namespace hinqs;
  if (!G || !theta_y)
    return fail(HINQS_ERR_ARG, "hinqs_selftest_projected_eig: NULL G or theta_y");
  if (m < 1 || m > kMaxSub)
    return fail(HINQS_ERR_ARG, "hinqs_selftest_projected_eig: m outside 1..%d", kMaxSub);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t mat = (size_t)kMaxSub * kMaxSub;
  std::vector<double> hg(mat, 0.0), hs(mat, 0.0);
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < m; ++c) {
      hg[(size_t)r * kMaxSub + c] = G[(size_t)r * m + c];
      if (S) hs[(size_t)r * kMaxSub + c] = S[(size_t)r * m + c];
    }
  double *dg = nullptr, *ds = nullptr, *dout = nullptr, *dall = nullptr;
  int* dpath = nullptr;
  int rc = HINQS_OK;
  if ((rc = dalloc(&dg, mat, s)) || (rc = dalloc(&ds, mat, s)) ||
      (rc = dalloc(&dout, (size_t)kRitzStride, s)) ||
      (rc = dalloc(&dall, (size_t)kMaxSub * kRitzStride, s)) || (rc = dalloc(&dpath, 1, s))) {
  }
  std::vector<double> hout(kRitzStride), hall((size_t)kMaxSub * kRitzStride);
  int hpath = 0;
  if (!rc) {
    cudaError_t e = cudaMemcpyAsync(dg, hg.data(), mat * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ds, hs.data(), mat * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      k_rr<<<1, kRRThreads, 0, s>>>(dg, kMaxSub, m, dout, S ? ds : nullptr, pairs ? dall : nullptr,
                                    nullptr, 0, dpath);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hout.data(), dout, hout.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hall.data(), dall, hall.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hpath, dpath, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "hinqs_selftest_projected_eig", __FILE__, __LINE__);
  }
  dfree(dg, s);
  dfree(ds, s);
  dfree(dout, s);
  dfree(dall, s);
  dfree(dpath, s);
  if (rc) return rc;
  for (int i = 0; i <= m; ++i) theta_y[i] = hout[i];
  if (pairs)
    for (int j = 0; j < m; ++j)
      for (int i = 0; i <= m; ++i) pairs[(size_t)j * (m + 1) + i] = hall[(size_t)j * kRitzStride + i];
  if (path) *path = hpath;
  return HINQS_OK;
}
