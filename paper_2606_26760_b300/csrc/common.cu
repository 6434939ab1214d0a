// Error plumbing, version, and the prepared Hamiltonian handle.
#include <cstdarg>
#include <cstring>

#include "hinqs_internal.cuh"

namespace hinqs {

static thread_local char g_err[1024] = "no error";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
  return HINQS_ERR_CUDA;
}

int smem_optin_limit() {
  static int cached[64] = {0};  // per device; a racing first fill writes the same value
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
      v = 227 * 1024;
    cached[dev] = v;
  }
  return cached[dev];
}

// FP64 -> FP32 copy (round to nearest).
__global__ void k_to_f32(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// Symmetry check: counts violations of h_pq = h_qp and of the 8-fold eri symmetry.
__global__ void k_check_sym(const double* __restrict__ h, const double* __restrict__ eri, int n,
                            unsigned int* bad) {
  int64_t n2 = (int64_t)n * n, n4 = n2 * n2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    int s = (int)(i % n), r = (int)((i / n) % n), q = (int)((i / n2) % n), p = (int)(i / (n2 * n));
    double v = eri[i];
    double tol = 1e-12 * (fabs(v) + 1e-300) + 1e-14;
    auto at = [&](int a, int b, int c, int d) { return eri[((int64_t)(a * n + b) * n + c) * n + d]; };
    if (fabs(at(q, p, r, s) - v) > tol || fabs(at(p, q, s, r) - v) > tol ||
        fabs(at(r, s, p, q) - v) > tol)
      atomicAdd(bad, 1u);
    if (i < n2) {
      int a = (int)(i / n), b = (int)(i % n);
      double x = h[i], y = h[b * n + a];
      if (fabs(x - y) > 1e-12 * (fabs(x) + 1e-300) + 1e-14) atomicAdd(bad, 1u);
    }
  }
}

}  // namespace hinqs

using namespace hinqs;

extern "C" const char* hinqs_last_error_message(void) { return g_err; }
extern "C" const char* hinqs_version(void) { return "hinqs-b300 0.1 (sm_103a)"; }

extern "C" int hinqs_ham_create(const double* h, const double* eri, int n_orb, int n_alpha,
                                int n_beta, double e_nuc, int flags, hinqs_ham** out,
                                void* stream) {
  if (!out) return fail(HINQS_ERR_ARG, "hinqs_ham_create: out is NULL");
  *out = nullptr;
  if (!h || !eri) return fail(HINQS_ERR_ARG, "hinqs_ham_create: h or eri is NULL");
  if (n_orb < 1 || n_orb > 64)
    return fail(HINQS_ERR_ARG, "hinqs_ham_create: n_orb=%d outside 1..64", n_orb);
  if (n_alpha < 0 || n_beta < 0 || n_alpha > n_orb || n_beta > n_orb)
    return fail(HINQS_ERR_ARG, "hinqs_ham_create: electron counts (%d,%d) outside 0..%d",
                n_alpha, n_beta, n_orb);
  cudaStream_t s = (cudaStream_t)stream;
  int64_t n2 = (int64_t)n_orb * n_orb, n4 = n2 * n2;
  if (flags & HINQS_CHECK_SYMMETRY) {
    unsigned int* bad = nullptr;
    HQ_TRY(dalloc(&bad, 1, s));
    HQ_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned int), s));
    k_check_sym<<<(int)std::min<int64_t>(ceil_div(n4, 256), 4096), 256, 0, s>>>(h, eri, n_orb, bad);
    unsigned int hb = 0;
    cudaError_t e = cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(bad, s);
    if (e != cudaSuccess) return cuda_fail(e, "symmetry check", __FILE__, __LINE__);
    if (hb) return fail(HINQS_ERR_ASYMMETRIC, "hinqs_ham_create: %u symmetry violations", hb);
  }
  hinqs_ham_s* H = new hinqs_ham_s();
  H->n = n_orb;
  H->n_alpha = n_alpha;
  H->n_beta = n_beta;
  H->e_nuc = e_nuc;
  int rc = HINQS_OK;
  if ((rc = dalloc(&H->h, n2, s)) || (rc = dalloc(&H->eri, n4, s)) ||
      (rc = dalloc(&H->h32, n2, s)) || (rc = dalloc(&H->eri32, n4, s))) {
    hinqs_ham_destroy(H);
    return rc;
  }
  cudaMemcpyAsync(H->h, h, n2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(H->eri, eri, n4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
  k_to_f32<<<(int)std::min<int64_t>(ceil_div(n2, 256), 1024), 256, 0, s>>>(H->h, H->h32, n2);
  k_to_f32<<<(int)std::min<int64_t>(ceil_div(n4, 256), 4096), 256, 0, s>>>(H->eri, H->eri32, n4);
  if ((rc = tc_tables_build(H, s)) < 0) {
    hinqs_ham_destroy(H);
    return rc;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    hinqs_ham_destroy(H);
    return cuda_fail(e, "hinqs_ham_create", __FILE__, __LINE__);
  }
  *out = H;
  return HINQS_OK;
}

extern "C" int hinqs_ham_destroy(hinqs_ham* H) {
  if (!H) return HINQS_OK;
  cudaStream_t s = 0;
  cudaDeviceSynchronize();
  dfree(H->h, s);
  dfree(H->eri, s);
  dfree(H->h32, s);
  dfree(H->eri32, s);
  dfree(H->tc_bhi, s);
  dfree(H->tc_blo, s);
  dfree(H->tc_bfold, s);
  delete H;
  return HINQS_OK;
}
