// Internal declarations of the HI-NQS B300 library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/hinqs.h"

namespace hinqs {

// ------------------------------------------------------------------ errors --
void set_error(const char* fmt, ...);
int fail(int code, const char* fmt, ...);  // records the message, returns code
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define HQ_CUDA(...)                                                       \
  do {                                                                     \
    cudaError_t e_ = (__VA_ARGS__);                                        \
    if (e_ != cudaSuccess) return hinqs::cuda_fail(e_, #__VA_ARGS__, __FILE__, __LINE__); \
  } while (0)

#define HQ_LAUNCH_CHECK() HQ_CUDA(cudaGetLastError())

#define HQ_TRY(...)                 \
  do {                              \
    int rc_ = (__VA_ARGS__);        \
    if (rc_ < 0) return rc_;        \
  } while (0)

// Stream-ordered device allocation from the default pool.
template <typename T>
int dalloc(T** p, size_t count, cudaStream_t s) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(HINQS_ERR_OOM, "device allocation of %zu bytes failed: %s", count * sizeof(T),
                cudaGetErrorString(e));
  }
  return HINQS_OK;
}

template <typename T>
void dfree(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync((void*)p, s);
  p = nullptr;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers
// (about 48 significant bits).  FP64 runs at 1/64 of the FP32 rate on this part and a
// double-float multiply-add is about twelve FP32 operations.  Products are exact up to
// the dropped lo*lo term (the error-free product by fused multiply-add), sums use the
// two-sum of Knuth, so each accumulated term carries about 2^-44 relative error.

// (sh, sl) += (ah + al) * (bh + bl)
__device__ __forceinline__ void df_fma(float ah, float al, float bh, float bl, float& sh,
                                       float& sl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float t = sh + p;
  const float z = t - sh;
  const float err = (sh - (t - z)) + (p - z);
  sh = t;
  sl += err + e;
}

// (sh, sl) += (bh, bl)
__device__ __forceinline__ void df_add(float bh, float bl, float& sh, float& sl) {
  const float t = sh + bh;
  const float z = t - sh;
  const float err = (sh - (t - z)) + (bh - z);
  sh = t;
  sl += err + bl;
}

__device__ __forceinline__ float2 df_split(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

constexpr int kNumSMs = 148;

}  // namespace hinqs

// ------------------------------------------------------------- handles ------

// Prepared Hamiltonian: copies of the FP64 integrals plus FP32 copies.
struct hinqs_ham_s {
  int n = 0, n_alpha = 0, n_beta = 0;
  double e_nuc = 0.0;
  double* h = nullptr;      // [n][n]
  double* eri = nullptr;    // [n*n][n*n] chemist (pq|rs), row pq, column rs
  float* h32 = nullptr;
  float* eri32 = nullptr;
  // tensor-core operand rows (n <= kTcMaxOrb): BF16 hi/lo of (pq|rs) over the folded
  // pairs r >= s, [n*n][8*tc_KB], zero-padded
  uint16_t* tc_bhi = nullptr;
  uint16_t* tc_blo = nullptr;
  int tc_KB = 0;
  // the whole folded table as the stationary B operand of the tile-stationary kernel
  // (n <= 22): rows = folded pairs pq, columns = folded pairs rs, Kp = tc_KB * 8 of
  // each, stored as the shared-memory image of a K-major core-matrix tile
  uint16_t* tc_bfold = nullptr;
};

constexpr int kTcMaxOrb = 32;
// sigma_ab_tc_launch: the operand tiles do not fit in shared memory (internal code;
// the caller computes the opposite-spin term on CUDA cores instead)
constexpr int kTcNoFit = 100;

// Sorted unique alpha and beta strings of the product subspace.
struct hinqs_subspace_s {
  int n = 0, n_alpha = 0, n_beta = 0;
  int64_t Na = 0, Nb = 0;
  uint64_t* sa = nullptr;  // [Na] ascending
  uint64_t* sb = nullptr;  // [Nb] ascending
};

// Same-spin string links of one spin species plus per-string tables.
//  all links (singles + doubles, ascending J per row):
//    row_ptr[N+1], col[nnz], hval64/hval32[nnz] (same-spin matrix element),
//    exc[nnz] packed p | q<<8 | r<<16 | s<<24 (r = s = 255 for singles),
//    sign[nnz], degree[nnz]
//  single links (ascending J per row): srow_ptr[N+1], slink[nsingle] = {J, signed pair}
//    with signed pair = sign * (p*n + q + 1)
//  per-string tables: hdiag[N] = H_spin(I,I) (FP64);
//    V64/V32[N][n*n] = sum_{i in I} (ii|xy), VT64/VT32 its transpose [n*n][N]
struct hinqs_links_s {
  int spin = 0, n = 0, n_e = 0;
  int64_t N = 0, nnz = 0, nsingle = 0;
  int max_row = 0, max_srow = 0;
  const uint64_t* strings = nullptr;  // borrowed from the subspace
  int64_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  double* hval64 = nullptr;
  float* hval32 = nullptr;
  uint32_t* exc = nullptr;
  int8_t* sign = nullptr;
  int8_t* degree = nullptr;
  int64_t* srow_ptr = nullptr;
  int2* slink = nullptr;
  double* hdiag = nullptr;
  double* V64 = nullptr;
  float* V32 = nullptr;
  double* VT64 = nullptr;  // [n*n][N], transpose of V
  float* VT32 = nullptr;
  float* VTlo32 = nullptr;  // fp32(VT64 - VT32): VT as a double-float pair with VT32
  // single links plus the n_e diagonal pseudo-links (J = I, pair jj, +1) of every
  // row, slot-major: sell[slot * N + I] = {J, sign * (pair + 1)}, slot < scount[I]
  int ell_width = 0;
  int2* sell = nullptr;
  int* scount = nullptr;
  // the same slots for the tensor-core gather: {J, kpart | (sign < 0) << 31} with kpart
  // the byte offset of the folded pair kf = max(p,q)(max(p,q)+1)/2 + min(p,q) inside a
  // K-major core-matrix row, (kf / 8) * 128 + (kf % 8) * 2; pair-major, slot k of row
  // I at ((k / 2) * N + I) * 2 + k % 2, so one 16-byte load brings two slots
  int2* tcell = nullptr;
  // the same slots packed into 32 bits, J | kpart << 17 | (sign < 0) << 31, quad-major:
  // slot k of row I at ((k / 4) * N + I) * 4 + k % 4, so one 16-byte load brings four
  // (kpart < 2^14 for n <= kTcMaxOrb); null when N > 2^17 or n > kTcMaxOrb
  uint32_t* tcq = nullptr;
  // all links as packed records for the row products: element offset of the linked
  // row (J * other dimension, uint32) with the element: rec32 {off, float bits},
  // rec64 {off, 0, double bits}; null when N_a * N_b >= 2^32
  int2* rec32 = nullptr;
  int4* rec64 = nullptr;
  // the same records for the BF16 copy of the operand (HINQS_PREC_FP32_BF16C), whose
  // rows are padded to ld16 = the other dimension rounded up to 64 elements (128-byte
  // rows): {J * ld16, float bits}; null when N * ld16 >= 2^32
  int2* rec16 = nullptr;
  int64_t ld16 = 0;
  // sigma tiles chosen by hinqs_autotune (0 = built-in default): rows per warp of
  // the row products that use these links, and the alpha-single chunk width of the
  // CUDA-core opposite-spin kernel (read from the alpha links)
  int tune_rows = 0;
  int tune_ch = 0;
  int tune_stages = 0;  // tensor-core pipeline depth (1 or 2; 0 = deepest that fits)
};

// A basis list of determinants inside a product subspace (Step 3's H_B over the
// list): entries sorted by product position I = i_a * N_b + i_b, distinct.
//   pos[m]     product positions, ascending
//   ia[m], ib[m]  string indices of each entry
//   arow[N_a+1]   entries of alpha string a are [arow[a], arow[a+1]), ascending in ib
struct hinqs_detlist_s {
  int64_t m = 0, Na = 0, Nb = 0;
  const uint64_t* sa = nullptr;  // borrowed from the subspace
  const uint64_t* sb = nullptr;
  int64_t* pos = nullptr;
  int32_t* ia = nullptr;
  int32_t* ib = nullptr;
  int64_t* arow = nullptr;
};

namespace hinqs {

// From this many determinants on, a problem's own (tuned) launches fill the GPU and
// it leaves the batched launches (measured on B300 with the 16-orbital (5,5) bond scan,
// sigma alone: batched 4.4x faster at 1e4 determinants per problem, 1.7x at 1.6e5,
// 1.2x at 6.4e5, 1.1x at 2.3e6, 0.94x at 6.3e6; within a solve the rendezvous of the
// rounds costs more than 1.1x gains).
constexpr int64_t kBatchSoloN = 1 << 20;

// Kernel launchers shared between translation units.
constexpr int kSameSpin = 1;      // H_a C + C H_b^T + diagonal + alpha-self x beta singles
constexpr int kOppositeSpin = 2;  // += alpha singles x (beta singles + beta self)
int sigma_launch(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                 const hinqs_links_s* lb, const void* c, void* sigma, int precision,
                 cudaStream_t s, int parts = kSameSpin | kOppositeSpin);
int diag_launch(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                const hinqs_links_s* lb, double* hdiag, cudaStream_t s);
// the same two operations on the determinants of a basis list (vectors of length m);
// list precision: HINQS_PREC_FP64, or FP32 for every FP32 mode
int sigma_list_launch(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                      const hinqs_links_s* lb, const hinqs_detlist_s* L, const void* c,
                      void* sigma, int precision, cudaStream_t s);
int diag_list_launch(const hinqs_ham_s* H, const hinqs_links_s* la, const hinqs_links_s* lb,
                     const hinqs_detlist_s* L, double* hdiag, cudaStream_t s);
int check_list(const hinqs_subspace_s* B, const hinqs_detlist_s* L, const char* who);
// One sigma product of a batch: y = H x for problem (H, B, la, lb) in `precision`.
struct SigmaReq {
  const hinqs_ham_s* H;
  const hinqs_subspace_s* B;
  const hinqs_links_s* la;
  const hinqs_links_s* lb;
  const void* x;
  void* y;
  int precision;
};
// The sigma products of several problems at once: FP32-family products run their
// same-spin stages and their tensor-core opposite-spin term as one launch per stage over
// all of them (a device work queue of (problem, alpha string) items for the tensor-core
// term); FP64 products, and those outside the batched kernels' range, run one by one.
int sigma_batch_launch(const SigmaReq* reqs, int n, cudaStream_t s);
// tensor-core opposite-spin term of the requests reqs[idx[0..n)] (split 1 or 3) in one
// launch; kTcNoFit when the batch cannot run as one launch (the caller runs them singly)
int sigma_ab_tc_batch(const SigmaReq* reqs, const int* idx, int n, int split, cudaStream_t s);
// Lockstep batching of Davidson solves (batch.cu): a solver with a batcher hands its
// sigma products to it, and each round's products run as one batched launch.
struct SigmaBatcher;
int batcher_sigma(SigmaBatcher* b, const SigmaReq& r, cudaStream_t s, cudaEvent_t ready);
// hinqs_davidson / hinqs_davidson_list with an optional batcher (davidson.cu)
int davidson_run(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                 const hinqs_links_s* lb, const hinqs_detlist_s* L, const double* guess,
                 const hinqs_davidson_opts* opts, double* energy, double* c_out,
                 hinqs_davidson_info* info_out, void* stream, const char* who,
                 SigmaBatcher* batcher, cudaEvent_t ready);
// opposite-spin sigma term on the tensor cores (FP32 vectors; split = 1 or 3)
int sigma_ab_tc_launch(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                       const hinqs_links_s* lb, const float* c, float* sig, int split,
                       cudaStream_t s);
// HINQS_ERR_TIMEOUT (and clears the flag) if a tensor-core kernel's bounded wait ran out
int tc_error_check(cudaStream_t s);
int tc_tables_build(hinqs_ham_s* H, cudaStream_t s);

// Opt-in shared-memory limit of the current device (bytes per block).
int smem_optin_limit();
// Raise a kernel's dynamic shared-memory cap to the device's opt-in limit.  The cap
// is a property of the kernel shared by every host thread, so it is always set to
// the same value: a per-launch value would race between concurrent solves.
// The carveout preference asks for the largest shared-memory split of the unified
// L1/shared storage, so that several large-tile CTAs can be resident on one SM.
// The cap is the opt-in limit less the kernel's static shared memory.
template <typename K>
int allow_max_smem(K kern) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_optin_limit() - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  return e == cudaSuccess ? HINQS_OK : cuda_fail(e, "cudaFuncSetAttribute", __FILE__, __LINE__);
}

}  // namespace hinqs

namespace hinqs {
// Spin-marginal reduction kernels (defined with hinqs_spin_marginals).
__global__ void k_row_sq(const double* __restrict__ C, int64_t Na, int64_t Nb, double* pa);
__global__ void k_col_sq(const double* __restrict__ C, int64_t Na, int64_t Nb, int64_t rows_per,
                         double* part);
__global__ void k_sum_chunks(const double* __restrict__ part, int64_t chunks, int64_t Nb, double* pb);
__global__ void k_marg_norm(double* pa, int64_t Na, double* pb, int64_t Nb, double* tot);
__global__ void k_teacher(const double* __restrict__ pa, const double* __restrict__ pb, int64_t Na,
                          int64_t Nb, const double* __restrict__ tot, double* __restrict__ w);

// Exclusive prefix sum of n int64 values on the device (out may alias in).
// If total != nullptr the grand total is copied to *total (host) after a
// stream synchronisation.
int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total,
                       cudaStream_t s);
// ascending bitonic sort of a[m_pad] in place (m_pad a power of two >= 2)
int bitonic_sort(uint64_t* a, int64_t m_pad, cudaStream_t s);
// the distinct strings of in[m] with k electrons in n orbitals, ascending, into a new
// device array *out (*count entries; *dropped strings failed the filter); HINQS_ERR_EMPTY
// when none is left (flags: HINQS_ERROR_BAD, HINQS_FULL_SPACE as hinqs_build_subspace)
int build_species(const uint64_t* in, int64_t m, int n, int k, int flags, uint64_t** out,
                  int64_t* count, int64_t* dropped, cudaStream_t s);
// Exact top-k selection (radix selection on order-preserving 64-bit keys): positions
// of the k entries of c[N] with the largest |c| (kSelAbs), the largest value
// (kSelLargest) or the smallest value (kSelSmallest), ties to the lower position,
// written ascending to out[min(k, N)].  Synchronises the stream.
constexpr int kSelAbs = 0, kSelLargest = 1, kSelSmallest = 2;
int select_top_impl(const double* c, int64_t N, int64_t k, int mode, int64_t* out,
                    cudaStream_t s);
}  // namespace hinqs
