// Measurement probe: the fused multiply-add rate of this GPU's FP64 and FP32 pipes.
//
// The bench reports the CUDA-core kernels of the sigma product (FP64 products,
// FP32 row products) against the rate of the unit that bounds them.  The driver
// measures only the copy bandwidth and the BF16 tensor rate, so this kernel measures
// the FMA rate itself: every SM runs resident warps whose threads each advance
// kChains independent FMA recurrences x <- x * a + b for `iters` steps (no memory
// traffic inside the loop; the chains are independent so the pipe, not the latency
// of one FMA, is the limit).  The result is written only when a run-time flag that
// the host never sets is true, which keeps the compiler from removing the chains.
#include <algorithm>

#include "hinqs_internal.cuh"

namespace hinqs {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(int iters, T a, T b, int store, T* out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (store) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static int fma_rate(double* tflops, cudaStream_t s) {
  int dev = 0, sms = kNumSMs, per_sm = 0;
  HQ_CUDA(cudaGetDevice(&dev));
  HQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_rate<T>, 256, 0));
  const int blocks = sms * std::max(per_sm, 1);
  const int iters = sizeof(T) == 8 ? 1 << 12 : 1 << 16;
  // a contraction that stays finite for any iteration count: |a| < 1
  const T a = (T)0.999999, b = (T)1e-6;
  cudaEvent_t e0, e1;
  HQ_CUDA(cudaEventCreate(&e0));
  HQ_CUDA(cudaEventCreate(&e1));
  k_fma_rate<T><<<blocks, 256, 0, s>>>(iters, a, b, 0, nullptr);  // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(e0, s);
    k_fma_rate<T><<<blocks, 256, 0, s>>>(iters, a, b, 0, nullptr);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HQ_LAUNCH_CHECK();
  const double flops = 2.0 * kChains * (double)iters * blocks * 256;
  *tflops = flops / (best * 1e-3) / 1e12;
  return HINQS_OK;
}

}  // namespace hinqs

extern "C" int hinqs_probe_fma_rate(int precision, double* tflops, void* stream) {
  if (!tflops) return hinqs::fail(HINQS_ERR_ARG, "hinqs_probe_fma_rate: tflops is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == HINQS_PREC_FP64) return hinqs::fma_rate<double>(tflops, s);
  if (precision == HINQS_PREC_FP32) return hinqs::fma_rate<float>(tflops, s);
  return hinqs::fail(HINQS_ERR_ARG, "hinqs_probe_fma_rate: precision must be FP64 or FP32");
}
