// Device exclusive prefix sum (three passes: block sums, scan of block sums,
// block-local scans plus offsets).
#include "hinqs_internal.cuh"

namespace hinqs {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
  __shared__ int64_t warp_sums[kScanThreads / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = w;
  }
  __syncthreads();
  int64_t incl = x + (wid > 0 ? warp_sums[wid - 1] : 0);
  if (total) *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return incl - v;
}

__global__ void k_scan_tile_sums(const int64_t* __restrict__ in, int64_t n, int64_t* sums) {
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t acc = 0;
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) acc += in[i];
  }
  int64_t tot;
  block_exclusive_scan(acc, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int64_t* sums, int64_t m, int64_t* grand) {
  // one block scans all tile sums in chunks
  int64_t carry = 0;
  for (int64_t base = 0; base < m; base += kScanThreads) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < m ? sums[i] : 0;
    int64_t tot;
    int64_t ex = block_exclusive_scan(v, &tot);
    if (i < m) sums[i] = ex + carry;
    carry += tot;
  }
  if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_apply(const int64_t* __restrict__ in, int64_t* out, int64_t n,
                             const int64_t* __restrict__ sums) {
  // each thread owns kScanItems consecutive elements
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t acc = 0;
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    acc += v[k];
  }
  int64_t tot;
  int64_t ex = block_exclusive_scan(acc, &tot) + sums[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
}

int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total,
                       cudaStream_t s) {
  if (n <= 0) {
    if (total) *total = 0;
    return HINQS_OK;
  }
  int64_t tiles = ceil_div(n, kScanTile);
  int64_t* sums = nullptr;
  HQ_TRY(dalloc(&sums, tiles + 1, s));
  k_scan_tile_sums<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums);
  k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, tiles, sums + tiles);
  k_scan_apply<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, sums);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && total) {
    e = cudaMemcpyAsync(total, sums + tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  dfree(sums, s);
  if (e != cudaSuccess) return cuda_fail(e, "exclusive_scan_i64", __FILE__, __LINE__);
  return HINQS_OK;
}

}  // namespace hinqs
