// Step 1' (Eq. classical_expansion) on the device: the determinants outside the
// product subspace that are connected by a non-zero Hamiltonian element to one of
// the n_top basis determinants with the largest |c_I|.
//
//  (1) Largest amplitudes: radix selection over the bit patterns of |c| (monotone
//      for non-negative doubles), eight bits per pass, then a stable compaction, so
//      the choice is exact and ties go to the lower index.
//  (2) Enumeration: one thread per (selected determinant, excitation): alpha and beta
//      singles and doubles and alpha-single x beta-single pairs, each with its
//      Slater-Condon element; kept when the element is non-zero and the result lies
//      outside S_alpha x S_beta, written as the key alpha << 32 | beta (n_orb < 32;
//      above, as the strings' ranks among the distinct kept strings), else a
//      sentinel.  Every slot is written once: no atomics, a deterministic set.
//  (3) Bitonic sort of the keys and a compaction of the distinct ones: candidates
//      ascending in (alpha, beta).
#include <algorithm>

#include "hinqs_internal.cuh"
#include "slater.cuh"

namespace hinqs {

namespace {

using namespace slater;
constexpr uint64_t kNoKey = ~0ull;

__device__ __forceinline__ uint64_t abs_bits(double x) {
  return (uint64_t)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// Selection key whose unsigned order is the wanted order of the values:
//   kSelAbs       |x| (its bit pattern is monotone for non-negative doubles);
//   kSelLargest   x itself: positive patterns get the top bit set, negative patterns
//                 are inverted, so the key increases with x (-0 is read as +0);
//   kSelSmallest  the complement of that, so the smallest x has the largest key.
// A NaN gets key 0 in the last two modes, below every number.
__device__ __forceinline__ uint64_t sel_key(double x, int mode) {
  if (mode == kSelAbs) return abs_bits(x);
  if (x != x) return 0ull;
  uint64_t u = (uint64_t)__double_as_longlong(x);
  if ((u << 1) == 0ull) u = 0ull;  // -0 -> +0
  const uint64_t ord = (u >> 63) ? ~u : (u | 0x8000000000000000ull);
  return mode == kSelLargest ? ord : ~ord;
}

// 256-bin histogram of bits [shift, shift+8) over the entries whose higher bits equal
// `prefix` under `mask`
__global__ void k_radix_hist(const double* __restrict__ c, int64_t N, int mode, uint64_t prefix,
                             uint64_t mask, int shift, unsigned long long* __restrict__ hist) {
  __shared__ unsigned int h[256];
  for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t u = sel_key(c[i], mode);
    if ((u & mask) == prefix) atomicAdd(&h[(u >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 256; b += blockDim.x)
    if (h[b]) atomicAdd(hist + b, (unsigned long long)h[b]);
}

// flag[i] = key of c_i above the threshold key (equal = 0) or equal to it (equal = 1)
__global__ void k_flag_key(const double* __restrict__ c, int64_t N, int mode, uint64_t key,
                           int equal, int64_t* __restrict__ flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t u = sel_key(c[i], mode);
    flag[i] = equal == 0 ? (u > key) : (u == key);
  }
}

// out[pos_gt[i] + ...]: indices above the threshold, plus the first `ties` equal ones,
// merged in ascending index order: rank = (#greater before i) + min(#equal before i, ties)
__global__ void k_select_scatter(const double* __restrict__ c, int64_t N, int mode, uint64_t key,
                                 int64_t ties, const int64_t* __restrict__ pos_gt,
                                 const int64_t* __restrict__ pos_eq, int64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t u = sel_key(c[i], mode);
    const bool take = u > key || (u == key && pos_eq[i] < ties);
    if (take) out[pos_gt[i] + std::min(pos_eq[i], ties)] = i;
  }
}

__device__ __forceinline__ int nth_set(uint64_t x, int k) {
  for (int i = 0; i < k; ++i) x &= x - 1;
  return __ffsll((long long)x) - 1;
}

// pair index t in [0, C(m, 2)) -> (i < j) in lexicographic order
__device__ __forceinline__ void unrank_pair(int m, int64_t t, int& i, int& j) {
  i = 0;
  while (t >= m - 1 - i) {
    t -= m - 1 - i;
    ++i;
  }
  j = i + 1 + (int)t;
}

struct ExpArgs {
  int n, na, nb;
  const double* h;
  const double* eri;
  const uint64_t* sa;
  const uint64_t* sb;
  int64_t Na, Nb;
  const int64_t* top;
  int64_t n_top;
  int64_t s1a, s1b, d2a, d2b, per;  // excitation counts per determinant
  uint64_t* keys;
  uint64_t* keys_b;  // n_orb >= 32: keys holds the alpha string, keys_b the beta string
  int64_t total;
  // basis list (list mode): only its determinants are left out, not the whole product
  const int64_t* arow;
  const int32_t* lib;
};

// is (i_a, i_b) an entry of the basis list (binary search in alpha string i_a's row)?
__device__ __forceinline__ bool in_list(const int64_t* __restrict__ arow,
                                        const int32_t* __restrict__ lib, int64_t a, int64_t b) {
  int64_t lo = arow[a], hi = arow[a + 1];
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    const int64_t v = lib[mid];
    if (v == b) return true;
    if (v < b) lo = mid + 1;
    else hi = mid;
  }
  return false;
}

__global__ void k_expand(ExpArgs A) {
  const uint64_t full = (1ull << A.n) - 1ull;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < A.total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = A.top[g / A.per];
    int64_t e = g % A.per;
    const uint64_t xa = A.sa[I / A.Nb], xb = A.sb[I % A.Nb];
    uint64_t ya = xa, yb = xb;
    double el = 0.0;
    const int va = A.n - A.na, vb = A.n - A.nb;
    if (e < A.s1a) {  // alpha single
      const int q = nth_set(xa, (int)(e / va)), p = nth_set(~xa & full, (int)(e % va));
      ya = (xa & ~(1ull << q)) | (1ull << p);
      el = single_elem(A.h, A.eri, A.n, xa, xb, p, q);
    } else if ((e -= A.s1a) < A.s1b) {  // beta single
      const int q = nth_set(xb, (int)(e / vb)), p = nth_set(~xb & full, (int)(e % vb));
      yb = (xb & ~(1ull << q)) | (1ull << p);
      el = single_elem(A.h, A.eri, A.n, xb, xa, p, q);
    } else if ((e -= A.s1b) < A.d2a) {  // alpha double
      const int64_t np = (int64_t)va * (va - 1) / 2;
      int h1, h2, p1, p2;
      unrank_pair(A.na, e / np, h1, h2);
      unrank_pair(va, e % np, p1, p2);
      const uint64_t holes = (1ull << nth_set(xa, h1)) | (1ull << nth_set(xa, h2));
      const uint64_t unocc = ~xa & full;
      const uint64_t parts = (1ull << nth_set(unocc, p1)) | (1ull << nth_set(unocc, p2));
      ya = (xa & ~holes) | parts;
      el = double_elem(A.eri, A.n, xa, ya);
    } else if ((e -= A.d2a) < A.d2b) {  // beta double
      const int64_t np = (int64_t)vb * (vb - 1) / 2;
      int h1, h2, p1, p2;
      unrank_pair(A.nb, e / np, h1, h2);
      unrank_pair(vb, e % np, p1, p2);
      const uint64_t holes = (1ull << nth_set(xb, h1)) | (1ull << nth_set(xb, h2));
      const uint64_t unocc = ~xb & full;
      const uint64_t parts = (1ull << nth_set(unocc, p1)) | (1ull << nth_set(unocc, p2));
      yb = (xb & ~holes) | parts;
      el = double_elem(A.eri, A.n, xb, yb);
    } else {  // alpha single x beta single
      e -= A.d2b;
      const int64_t ea = e / A.s1b, eb = e % A.s1b;
      const int qa = nth_set(xa, (int)(ea / va)), pa = nth_set(~xa & full, (int)(ea % va));
      const int qb = nth_set(xb, (int)(eb / vb)), pb = nth_set(~xb & full, (int)(eb % vb));
      ya = (xa & ~(1ull << qa)) | (1ull << pa);
      yb = (xb & ~(1ull << qb)) | (1ull << pb);
      el = single_sign(xa, pa, qa) * single_sign(xb, pb, qb) * eri4(A.eri, A.n, pa, qa, pb, qb);
    }
    const int64_t ya_i = find_string(A.sa, A.Na, ya);
    const int64_t yb_i = ya_i >= 0 ? find_string(A.sb, A.Nb, yb) : -1;
    bool inside = ya_i >= 0 && yb_i >= 0;
    if (inside && A.arow) inside = in_list(A.arow, A.lib, ya_i, yb_i);
    const bool keep = el != 0.0 && !inside;
    if (A.keys_b) {
      A.keys[g] = keep ? ya : kNoKey;
      A.keys_b[g] = keep ? yb : kNoKey;
    } else {
      A.keys[g] = keep ? ((ya << 32) | yb) : kNoKey;
    }
  }
}

__global__ void k_map_positions(int64_t* idx, int64_t k, const int64_t* __restrict__ pos) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k;
       i += (int64_t)gridDim.x * blockDim.x)
    idx[i] = pos[idx[i]];
}

__global__ void k_fill_key(uint64_t* a, int64_t from, int64_t to) {
  for (int64_t i = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < to;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = kNoKey;
}

__global__ void k_distinct_flags(const uint64_t* __restrict__ a, int64_t m, int64_t* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (a[i] != kNoKey && (i == 0 || a[i] != a[i - 1])) ? 1 : 0;
}

// DA / DB NULL: the key is alpha << 32 | beta; else ranks in the dictionaries
__global__ void k_split_keys(const uint64_t* __restrict__ a, int64_t m, const int64_t* pos,
                             const uint64_t* __restrict__ DA, const uint64_t* __restrict__ DB,
                             uint64_t* __restrict__ xa, uint64_t* __restrict__ xb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    if (a[i] != kNoKey && (i == 0 || a[i] != a[i - 1])) {
      const uint64_t hi = a[i] >> 32, lo = a[i] & 0xffffffffull;
      xa[pos[i]] = DA ? DA[hi] : hi;
      xb[pos[i]] = DB ? DB[lo] : lo;
    }
}

// n_orb >= 32: (alpha, beta) strings -> rank(alpha) << 32 | rank(beta) in place (keys
// holds alpha, keys_b beta; kNoKey stays kNoKey)
__global__ void k_rank_keys(uint64_t* __restrict__ keys, const uint64_t* __restrict__ keys_b,
                            int64_t m, const uint64_t* __restrict__ DA, int64_t ua,
                            const uint64_t* __restrict__ DB, int64_t ub) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = keys[i];
    if (a == kNoKey) continue;
    const int64_t ra = find_string(DA, ua, a), rb = find_string(DB, ub, keys_b[i]);
    keys[i] = (ra >= 0 && rb >= 0) ? (((uint64_t)ra << 32) | (uint64_t)rb) : kNoKey;
  }
}

}  // namespace

// the k entries of c with the largest selection key (mode: kSelAbs = largest |c|,
// kSelLargest, kSelSmallest; ties: lower index first), ascending indices, into out[k]
int select_top_impl(const double* c, int64_t N, int64_t k, int mode, int64_t* out,
                    cudaStream_t s) {
  k = std::min(k, N);
  if (k <= 0) return HINQS_OK;
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(N, 256), 8 * kNumSMs);
  unsigned long long* hist = nullptr;
  int64_t *f_gt = nullptr, *f_eq = nullptr;
  int rc = HINQS_OK;
  auto run = [&]() -> int {
    HQ_TRY(dalloc(&hist, 256, s));
    uint64_t prefix = 0, mask = 0;
    int64_t need = k;  // entries still to take at or below the current prefix
    for (int shift = 56; shift >= 0; shift -= 8) {
      HQ_CUDA(cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned long long), s));
      k_radix_hist<<<grid, 256, 0, s>>>(c, N, mode, prefix, mask, shift, hist);
      HQ_LAUNCH_CHECK();
      unsigned long long hh[256];
      HQ_CUDA(cudaMemcpyAsync(hh, hist, sizeof(hh), cudaMemcpyDeviceToHost, s));
      HQ_CUDA(cudaStreamSynchronize(s));
      int b = 255;
      for (; b > 0; --b) {
        if ((int64_t)hh[b] >= need) break;
        need -= (int64_t)hh[b];
      }
      prefix |= (uint64_t)b << shift;
      mask |= 255ull << shift;
    }
    // prefix is the k-th largest key; take every larger entry and `need` equal ones
    HQ_TRY(dalloc(&f_gt, N, s));
    HQ_TRY(dalloc(&f_eq, N, s));
    k_flag_key<<<grid, 256, 0, s>>>(c, N, mode, prefix, 0, f_gt);
    k_flag_key<<<grid, 256, 0, s>>>(c, N, mode, prefix, 1, f_eq);
    HQ_LAUNCH_CHECK();
    int64_t n_gt = 0, n_eq = 0;
    HQ_TRY(exclusive_scan_i64(f_gt, f_gt, N, &n_gt, s));
    HQ_TRY(exclusive_scan_i64(f_eq, f_eq, N, &n_eq, s));
    if (n_gt + std::min(n_eq, need) != k)
      return fail(HINQS_ERR_CUDA, "top amplitudes: selection count mismatch");
    k_select_scatter<<<grid, 256, 0, s>>>(c, N, mode, prefix, need, f_gt, f_eq, out);
    HQ_LAUNCH_CHECK();
    return HINQS_OK;
  };
  rc = run();
  dfree(hist, s);
  dfree(f_gt, s);
  dfree(f_eq, s);
  return rc;
}

}  // namespace hinqs

using namespace hinqs;

extern "C" int hinqs_top_amplitudes(const hinqs_subspace* B, const double* c, int64_t k,
                                    int64_t* idx_out, void* stream) {
  if (!B || !c || k < 0 || (k > 0 && !idx_out))
    return fail(HINQS_ERR_ARG, "hinqs_top_amplitudes: NULL argument or negative k");
  return select_top_impl(c, B->Na * B->Nb, k, kSelAbs, idx_out, (cudaStream_t)stream);
}

// Step 1' over the product (L = NULL: c over the product, the product left out) or over
// a basis list (c over the list entries, only the list left out)
static int expansion_impl(const hinqs_ham* H, const hinqs_subspace* B, const hinqs_detlist* L,
                          const double* c, int64_t n_top, uint64_t* xa_out, uint64_t* xb_out,
                          int64_t cap, int64_t* count, void* stream, const char* who) {
  if (!H || !B || !c || !count || n_top < 0)
    return fail(HINQS_ERR_ARG, "%s: NULL argument or negative n_top", who);
  if (H->n != B->n || H->n_alpha != B->n_alpha || H->n_beta != B->n_beta)
    return fail(HINQS_ERR_ARG, "%s: Hamiltonian and subspace disagree", who);
  if (L) HQ_TRY(check_list(B, L, who));
  if (H->n_alpha == 64 || H->n_beta == 64)
    return fail(HINQS_ERR_ARG, "%s: 64 electrons of one spin are not supported", who);
  *count = 0;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = L ? L->m : B->Na * B->Nb;
  n_top = std::min(n_top, N);
  if (n_top == 0) return HINQS_OK;
  ExpArgs A;
  A.n = H->n;
  A.na = H->n_alpha;
  A.nb = H->n_beta;
  A.h = H->h;
  A.eri = H->eri;
  A.sa = B->sa;
  A.sb = B->sb;
  A.Na = B->Na;
  A.Nb = B->Nb;
  A.arow = L ? L->arow : nullptr;
  A.lib = L ? L->ib : nullptr;
  const int64_t va = A.n - A.na, vb = A.n - A.nb;
  A.s1a = A.na * va;
  A.s1b = A.nb * vb;
  A.d2a = (int64_t)A.na * (A.na - 1) / 2 * (va * (va - 1) / 2);
  A.d2b = (int64_t)A.nb * (A.nb - 1) / 2 * (vb * (vb - 1) / 2);
  A.per = A.s1a + A.s1b + A.d2a + A.d2b + A.s1a * A.s1b;
  A.n_top = n_top;
  A.total = n_top * A.per;
  if (A.per == 0) return HINQS_OK;
  int64_t m_pad = 2;
  while (m_pad < A.total) m_pad <<= 1;
  // n_orb <= 31: keys alpha << 32 | beta; else ranks in the candidates' distinct strings
  const bool ranks = H->n >= 32;
  int64_t* top = nullptr;
  uint64_t *keys = nullptr, *keys_b = nullptr, *DA = nullptr, *DB = nullptr;
  int64_t* pos = nullptr;
  auto run = [&]() -> int {
    HQ_TRY(dalloc(&top, n_top, s));
    HQ_TRY(select_top_impl(c, N, n_top, kSelAbs, top, s));
    if (L) {  // list entries -> product positions
      k_map_positions<<<(unsigned)std::min<int64_t>(ceil_div(n_top, 256), 1024), 256, 0, s>>>(
          top, n_top, L->pos);
      HQ_LAUNCH_CHECK();
    }
    HQ_TRY(dalloc(&keys, m_pad, s));
    if (ranks) HQ_TRY(dalloc(&keys_b, A.total, s));
    A.top = top;
    A.keys = keys;
    A.keys_b = keys_b;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(m_pad, 256), 16 * kNumSMs);
    k_expand<<<grid, 256, 0, s>>>(A);
    k_fill_key<<<grid, 256, 0, s>>>(keys, A.total, m_pad);
    HQ_LAUNCH_CHECK();
    int64_t ua = 0, ub = 0;
    if (ranks) {
      // dictionaries of the kept alpha and beta strings (kNoKey fails the filter)
      int64_t drop = 0;
      int r = build_species(keys, A.total, A.n, A.na, 0, &DA, &ua, &drop, s);
      if (r < 0 && r != HINQS_ERR_EMPTY) return r;
      if (r == HINQS_ERR_EMPTY) return HINQS_OK;  // nothing kept
      r = build_species(keys_b, A.total, A.n, A.nb, 0, &DB, &ub, &drop, s);
      if (r < 0) return r;
      k_rank_keys<<<grid, 256, 0, s>>>(keys, keys_b, A.total, DA, ua, DB, ub);
      HQ_LAUNCH_CHECK();
    }
    HQ_TRY(bitonic_sort(keys, m_pad, s));
    HQ_TRY(dalloc(&pos, m_pad, s));
    k_distinct_flags<<<grid, 256, 0, s>>>(keys, m_pad, pos);
    HQ_LAUNCH_CHECK();
    int64_t uniq = 0;
    HQ_TRY(exclusive_scan_i64(pos, pos, m_pad, &uniq, s));
    *count = uniq;
    if (!xa_out || !xb_out) return HINQS_OK;  // count only
    if (cap < uniq)
      return fail(HINQS_ERR_ARG, "%s: cap %lld below the %lld candidates", who, (long long)cap,
                  (long long)uniq);
    k_split_keys<<<grid, 256, 0, s>>>(keys, m_pad, pos, DA, DB, xa_out, xb_out);
    HQ_LAUNCH_CHECK();
    return HINQS_OK;
  };
  const int rc = run();
  dfree(top, s);
  dfree(keys, s);
  dfree(keys_b, s);
  dfree(DA, s);
  dfree(DB, s);
  dfree(pos, s);
  return rc;
}

extern "C" int hinqs_classical_expansion(const hinqs_ham* H, const hinqs_subspace* B,
                                         const double* c, int64_t n_top, uint64_t* xa_out,
                                         uint64_t* xb_out, int64_t cap, int64_t* count,
                                         void* stream) {
  return expansion_impl(H, B, nullptr, c, n_top, xa_out, xb_out, cap, count, stream,
                        "hinqs_classical_expansion");
}

extern "C" int hinqs_classical_expansion_list(const hinqs_ham* H, const hinqs_subspace* B,
                                              const hinqs_detlist* L, const double* c_list,
                                              int64_t n_top, uint64_t* xa_out, uint64_t* xb_out,
                                              int64_t cap, int64_t* count, void* stream) {
  if (!L) return fail(HINQS_ERR_ARG, "hinqs_classical_expansion_list: NULL list");
  return expansion_impl(H, B, L, c_list, n_top, xa_out, xb_out, cap, count, stream,
                        "hinqs_classical_expansion_list");
}
