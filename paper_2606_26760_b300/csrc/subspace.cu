// K1: the SQD product subspace from sampled strings (particle-number filter,
// sort, unique) or the full space by combinatorial unranking.
#include <algorithm>

#include "hinqs_internal.cuh"

namespace hinqs {

constexpr uint64_t kSentinel = ~0ull;

// Invalid strings (wrong popcount or bits >= n) become the sentinel so they sort last.
__global__ void k_filter(const uint64_t* __restrict__ in, int64_t m, uint64_t* __restrict__ out,
                         int64_t m_pad, int n, int k, unsigned long long* bad) {
  uint64_t hi_mask = (n == 64) ? 0ull : (~0ull << n);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t v = kSentinel;
    if (i < m) {
      uint64_t x = in[i];
      if (__popcll(x) == k && (x & hi_mask) == 0) v = x;
      else atomicAdd(bad, 1ull);
    }
    out[i] = v;
  }
}

// One compare-exchange stage of a bitonic sorting network (ascending overall).
__global__ void k_bitonic_global(uint64_t* a, int64_t m_pad, int64_t j, int64_t k) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t l = i ^ j;
    if (l > i) {
      uint64_t x = a[i], y = a[l];
      bool up = (i & k) == 0;
      if ((x > y) == up) {
        a[i] = y;
        a[l] = x;
      }
    }
  }
}

// The stages with j < 1024 of one k, on a 2048-element tile in shared memory.
__global__ void k_bitonic_shared(uint64_t* a, int64_t k, int64_t j_start) {
  __shared__ uint64_t t[2048];
  int64_t base = (int64_t)blockIdx.x * 2048;
  t[threadIdx.x] = a[base + threadIdx.x];
  t[threadIdx.x + 1024] = a[base + threadIdx.x + 1024];
  __syncthreads();
  for (int64_t j = j_start; j > 0; j >>= 1) {
    for (int h = 0; h < 2; ++h) {
      int64_t i = threadIdx.x + h * 1024;
      int64_t l = i ^ j;
      if (l > i) {
        uint64_t x = t[i], y = t[l];
        bool up = ((base + i) & k) == 0;
        if ((x > y) == up) {
          t[i] = y;
          t[l] = x;
        }
      }
    }
    __syncthreads();
  }
  a[base + threadIdx.x] = t[threadIdx.x];
  a[base + threadIdx.x + 1024] = t[threadIdx.x + 1024];
}

int bitonic_sort(uint64_t* a, int64_t m_pad, cudaStream_t s) {
  int grid = (int)std::min<int64_t>(ceil_div(m_pad / 2, 256) + 1, 8 * kNumSMs);
  for (int64_t k = 2; k <= m_pad; k <<= 1) {
    int64_t j = k >> 1;
    for (; j > 0; j >>= 1) {
      if (j < 1024 && m_pad >= 2048) {
        k_bitonic_shared<<<(unsigned)(m_pad / 2048), 1024, 0, s>>>(a, k, j);
        break;
      }
      k_bitonic_global<<<grid, 256, 0, s>>>(a, m_pad, j, k);
    }
  }
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

__global__ void k_unique_flags(const uint64_t* __restrict__ a, int64_t m, int64_t* flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    flags[i] = (a[i] != kSentinel && (i == 0 || a[i] != a[i - 1])) ? 1 : 0;
}

__global__ void k_unique_scatter(const uint64_t* __restrict__ a, int64_t m,
                                 const int64_t* __restrict__ pos, uint64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    if (a[i] != kSentinel && (i == 0 || a[i] != a[i - 1])) out[pos[i]] = a[i];
}

// Binomial table binom[a*65+b] = C(a,b) for a, b <= 64 (saturating at ~0ull).
struct Binom {
  uint64_t c[65][65];
};

static void make_binom(Binom& B) {
  for (int a = 0; a <= 64; ++a)
    for (int b = 0; b <= 64; ++b) {
      if (b == 0) B.c[a][b] = 1;
      else if (a == 0) B.c[a][b] = 0;
      else {
        uint64_t x = B.c[a - 1][b - 1], y = B.c[a - 1][b];
        B.c[a][b] = (x > ~0ull - y) ? ~0ull : x + y;
      }
    }
}

uint64_t binom_host(int a, int b) {
  static Binom B;
  static bool init = false;
  if (!init) {
    make_binom(B);
    init = true;
  }
  if (a < 0 || b < 0 || b > a) return 0;
  return B.c[a][b];
}

// Colex unranking: ascending integer order of k-subsets equals colex order,
// rank = sum_i C(c_i, i) for elements c_1 < ... < c_k.
__global__ void k_unrank(uint64_t* out, int64_t count, int n, int k, const uint64_t* binom) {
  for (int64_t r0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r0 < count;
       r0 += (int64_t)gridDim.x * blockDim.x) {
    uint64_t r = (uint64_t)r0, v = 0;
    int c = n - 1;
    for (int i = k; i >= 1; --i) {
      while (c >= 0 && binom[c * 65 + i] > r) --c;
      v |= 1ull << c;
      r -= binom[c * 65 + i];
      --c;
    }
    out[r0] = v;
  }
}

int build_species(const uint64_t* in, int64_t m, int n, int k, int flags, uint64_t** out,
                         int64_t* count, int64_t* dropped, cudaStream_t s) {
  *out = nullptr;
  *count = 0;
  *dropped = 0;
  if (flags & HINQS_FULL_SPACE) {
    uint64_t total = binom_host(n, k);
    if (total == 0 || total > (uint64_t)INT32_MAX)
      return fail(HINQS_ERR_ARG, "full space C(%d,%d) is empty or exceeds 2^31-1 strings", n, k);
    static uint64_t* d_binom = nullptr;
    static int dev_of_binom = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (!d_binom || dev_of_binom != dev) {
      Binom B;
      make_binom(B);
      HQ_CUDA(cudaMalloc((void**)&d_binom, sizeof(Binom)));
      HQ_CUDA(cudaMemcpy(d_binom, &B, sizeof(Binom), cudaMemcpyHostToDevice));
      dev_of_binom = dev;
    }
    HQ_TRY(dalloc(out, total, s));
    k_unrank<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 8 * kNumSMs), 256, 0, s>>>(
        *out, (int64_t)total, n, k, d_binom);
    HQ_LAUNCH_CHECK();
    *count = (int64_t)total;
    return HINQS_OK;
  }
  if (m <= 0) return fail(HINQS_ERR_EMPTY, "no input strings");
  if (k == 64) return fail(HINQS_ERR_ARG, "64 electrons in 64 orbitals is not supported");
  int64_t m_pad = 1;
  while (m_pad < m) m_pad <<= 1;
  if (m_pad < 2048) m_pad = 2048;
  uint64_t* buf = nullptr;
  int64_t* pos = nullptr;
  unsigned long long* bad = nullptr;
  int rc = HINQS_OK;
  if ((rc = dalloc(&buf, m_pad, s)) || (rc = dalloc(&pos, m_pad, s)) || (rc = dalloc(&bad, 1, s))) {
    dfree(buf, s);
    dfree(pos, s);
    dfree(bad, s);
    return rc;
  }
  cudaMemsetAsync(bad, 0, sizeof(*bad), s);
  int grid = (int)std::min<int64_t>(ceil_div(m_pad, 256), 8 * kNumSMs);
  k_filter<<<grid, 256, 0, s>>>(in, m, buf, m_pad, n, k, bad);
  unsigned long long hbad = 0;
  int64_t uniq = 0;
  rc = bitonic_sort(buf, m_pad, s);
  if (!rc) {
    k_unique_flags<<<grid, 256, 0, s>>>(buf, m_pad, pos);
    rc = exclusive_scan_i64(pos, pos, m_pad, &uniq, s);
  }
  if (!rc) {
    cudaMemcpy(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost);
    *dropped = (int64_t)hbad;
    if (hbad && (flags & HINQS_ERROR_BAD))
      rc = fail(HINQS_ERR_PARTICLE_NUMBER, "%llu strings with the wrong particle number", hbad);
    else if (uniq == 0)
      rc = fail(HINQS_ERR_EMPTY, "no string with %d electrons in %d orbitals", k, n);
    else if (uniq > INT32_MAX)
      rc = fail(HINQS_ERR_ARG, "more than 2^31-1 unique strings");
  }
  if (!rc) rc = dalloc(out, uniq, s);
  if (!rc) {
    k_unique_scatter<<<grid, 256, 0, s>>>(buf, m_pad, pos, *out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "unique scatter", __FILE__, __LINE__);
    *count = uniq;
  }
  dfree(buf, s);
  dfree(pos, s);
  dfree(bad, s);
  if (rc) dfree(*out, s);
  return rc;
}

}  // namespace hinqs

using namespace hinqs;

extern "C" int hinqs_build_subspace(const uint64_t* alpha, int64_t n_a_in, const uint64_t* beta,
                                    int64_t n_b_in, int n_orb, int n_alpha, int n_beta, int flags,
                                    hinqs_subspace** out, int64_t* n_dropped, void* stream) {
  if (!out) return fail(HINQS_ERR_ARG, "hinqs_build_subspace: out is NULL");
  *out = nullptr;
  if (n_orb < 1 || n_orb > 64 || n_alpha < 0 || n_beta < 0 || n_alpha > n_orb || n_beta > n_orb)
    return fail(HINQS_ERR_ARG, "hinqs_build_subspace: bad sizes n_orb=%d n_alpha=%d n_beta=%d",
                n_orb, n_alpha, n_beta);
  if (!(flags & HINQS_FULL_SPACE) &&
      ((n_a_in > 0 && !alpha) || (n_b_in > 0 && !beta) || n_a_in < 0 || n_b_in < 0))
    return fail(HINQS_ERR_ARG, "hinqs_build_subspace: NULL or negative-size string arrays");
  cudaStream_t s = (cudaStream_t)stream;
  hinqs_subspace_s* B = new hinqs_subspace_s();
  B->n = n_orb;
  B->n_alpha = n_alpha;
  B->n_beta = n_beta;
  int64_t da = 0, db = 0;
  int rc = build_species(alpha, n_a_in, n_orb, n_alpha, flags, &B->sa, &B->Na, &da, s);
  if (!rc) rc = build_species(beta, n_b_in, n_orb, n_beta, flags, &B->sb, &B->Nb, &db, s);
  if (n_dropped) {
    n_dropped[0] = da;
    n_dropped[1] = db;
  }
  if (rc) {
    hinqs_subspace_destroy(B);
    return rc;
  }
  *out = B;
  return HINQS_OK;
}

extern "C" int hinqs_subspace_dims(const hinqs_subspace* B, int64_t* n_a, int64_t* n_b) {
  if (!B) return fail(HINQS_ERR_ARG, "hinqs_subspace_dims: NULL handle");
  if (n_a) *n_a = B->Na;
  if (n_b) *n_b = B->Nb;
  return HINQS_OK;
}

extern "C" int hinqs_subspace_strings(const hinqs_subspace* B, uint64_t* a, uint64_t* b,
                                      void* stream) {
  if (!B) return fail(HINQS_ERR_ARG, "hinqs_subspace_strings: NULL handle");
  cudaStream_t s = (cudaStream_t)stream;
  if (a) HQ_CUDA(cudaMemcpyAsync(a, B->sa, B->Na * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  if (b) HQ_CUDA(cudaMemcpyAsync(b, B->sb, B->Nb * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  return HINQS_OK;
}

extern "C" int hinqs_subspace_destroy(hinqs_subspace* B) {
  if (!B) return HINQS_OK;
  cudaDeviceSynchronize();
  dfree(B->sa, 0);
  dfree(B->sb, 0);
  delete B;
  return HINQS_OK;
}
