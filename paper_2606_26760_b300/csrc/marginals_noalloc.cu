// Spin marginals without any device allocation.
//
// Same result as hinqs_spin_marginals, but the reduction's scratch space (the
// per-chunk column partial sums and two scalars) lives in a fixed array in this
// file instead of memory obtained from cudaMallocAsync.  It serves callers that
// cannot allocate device memory while they run: a process whose allocator has
// already reserved the device memory it may use, or a serving loop that must not
// meet an out-of-memory failure, or change its memory footprint, once it is up.
//
// The array is a file-scope __device__ object, so every GPU that loads this
// library holds it (8 MiB) until the process exits.  Host code cannot use its
// name as a device address; the address is obtained once per device with
// cudaGetSymbolAddress, with that device current, by the first call on that
// device.  That first call therefore also runs the set-up and should come before
// any stream capture.  All calls share the one array: calls whose execution can
// overlap on the GPU (different streams, or different host threads) race on it
// and must be serialised by the caller.
#include <mutex>

#include "hinqs_internal.cuh"

namespace hinqs {

// Capacity in doubles: two scalars followed by the column partial sums.
constexpr int64_t kNoAllocScratch = int64_t(1) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_marginal_scratch[kNoAllocScratch];

static std::mutex g_scratch_mutex;
static double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set up on first use).
static int scratch_address(double** out) {
  int dev = 0;
  HQ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(HINQS_ERR_ARG, "hinqs_spin_marginals_noalloc: device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_marginal_scratch);
    if (e != cudaSuccess || !p)
      return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                       "cudaGetSymbolAddress(g_marginal_scratch)", __FILE__, __LINE__);
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return HINQS_OK;
}

}  // namespace hinqs

using namespace hinqs;

extern "C" int hinqs_spin_marginals_noalloc(const hinqs_subspace* B, const double* c, double* pa,
                                            double* pb, double* w, void* stream) {
  if (!B || !c || !pa || !pb)
    return fail(HINQS_ERR_ARG, "hinqs_spin_marginals_noalloc: NULL argument");
  const int64_t Na = B->Na, Nb = B->Nb;
  const int64_t cap = kNoAllocScratch - 2;  // doubles left for the column partial sums
  if (Nb > cap)
    return fail(HINQS_ERR_ARG,
                "hinqs_spin_marginals_noalloc: N_beta = %lld exceeds the fixed scratch of %lld "
                "doubles; use hinqs_spin_marginals",
                (long long)Nb, (long long)cap);
  double* scratch = nullptr;
  HQ_TRY(scratch_address(&scratch));
  double* tot = scratch;      // [2], written before it is read
  double* part = scratch + 2;  // [chunks][Nb], every entry written before it is read
  // as many row chunks as fit (each chunk adds Nb partial sums), at least 64 rows each,
  // and at most 65535 chunks (grid y limit)
  const int64_t max_chunks = std::min<int64_t>(cap / Nb, 65535);
  int64_t rows_per = std::max<int64_t>(64, ceil_div(Na, max_chunks));
  const int64_t chunks = ceil_div(Na, rows_per);
  cudaStream_t s = (cudaStream_t)stream;
  k_row_sq<<<(unsigned)std::min<int64_t>(Na, 16 * kNumSMs), 256, 0, s>>>(c, Na, Nb, pa);
  dim3 g((unsigned)std::min<int64_t>(ceil_div(Nb, 256), 64), (unsigned)chunks);
  k_col_sq<<<g, 256, 0, s>>>(c, Na, Nb, rows_per, part);
  k_sum_chunks<<<(unsigned)std::min<int64_t>(ceil_div(Nb, 256), 256), 256, 0, s>>>(part, chunks, Nb,
                                                                                   pb);
  k_marg_norm<<<1, 1024, 0, s>>>(pa, Na, pb, Nb, tot);
  if (w)
    k_teacher<<<(unsigned)std::min<int64_t>(ceil_div(Na * Nb, 256), 16 * kNumSMs), 256, 0, s>>>(
        pa, pb, Na, Nb, tot, w);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}
