// K5 -> K6 -> K7 on the 5th-generation tensor cores: the opposite-spin part of
// sigma written as a gather into D followed by a dense GEMM against (pq|rs),
//
//   sigma(Ia,Ib) += sum_{alpha singles Ja -> Ia, pair pq, sign s_a} s_a E(Ja,Ib;pq),
//   E(Ja,Ib;pq)   = sum_rs (pq|rs) D(Ja,Ib;rs),
//   D(Ja,Ib;rs)   = sum_{beta singles Ib -> Jb with pair rs} s_b C(Ja,Jb)
//                   + [rs = jj, j in Ib] C(Ja,Ib).
//
// One CTA per alpha string Ja.  The (pq|rs) columns of Ja's alpha singles form
// the B operand [NW x K] and each tile of 128 beta strings forms the A operand
// D [128 x K], both BF16 in shared memory (K-major, canonical no-swizzle layout of
// 8x16-byte core matrices); K runs over the folded pairs r >= s (the integral is
// symmetric in r,s and a beta string contributes at most one of rs, sr), padded
// to a multiple of 16.  One thread issues the tcgen05.mma chain into an FP32
// accumulator in tensor memory; the four warps read their 32 lanes back with
// tcgen05.ld and add s_a E into sigma with coalesced atomics.
// SPLIT = 3 represents each operand as hi + lo BF16 terms and accumulates
// hi*hi + hi*lo + lo*hi (about 16 significant bits); SPLIT = 1 uses hi only.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "hinqs_internal.cuh"

namespace hinqs {

__device__ int g_tc_error = 0;  // set by a CTA whose bounded wait ran out

namespace tc {

constexpr int kThreads = 128;
constexpr int kTileM = 128;
constexpr long long kWaitLimit = 1ll << 26;  // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle: start >> 4, LBO >> 4
// (K-direction core-matrix stride), SBO >> 4 (8-row-group stride), version 1.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (r, k) in a K-major tile with KB 8-element K blocks
__device__ __forceinline__ uint32_t tile_off(int r, int k, int KB) {
  return (uint32_t)((r >> 3) * (KB * 128) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (long long it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

struct Args {
  int64_t Na, Nb;
  int n, K, KB;  // folded pairs, padded K / 8
  const int64_t* a_srow;
  const int2* a_slink;
  const int2* b_ell;
  const int* b_cnt;
  const float* eri;  // FP32 (pq|rs), [n2][n2]
  const float* C;
  float* sig;
  int crow_smem;  // stage the row C(Ja, :) in shared memory
  int vec4;       // N_b % 4 == 0: float4 atomics are aligned
};

__device__ __forceinline__ int fold_index(int r, int s) {
  if (r < s) {
    int t = r;
    r = s;
    s = t;
  }
  return r * (r + 1) / 2 + s;
}

template <int NW, int SPLIT>
__global__ void __launch_bounds__(kThreads, 1) k_sigma_ab_tc(Args A) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int KB = A.KB, Kp = KB * 8, n = A.n, n2 = n * n;
  // each A region also holds the [16][kTileM] FP32 epilogue staging, so at least 8 KB
  const uint32_t a_bytes = max((uint32_t)kTileM * Kp * 2, 16u * kTileM * 4u);
  const uint32_t b_bytes = (uint32_t)NW * Kp * 2;
  unsigned char* a_hi = smem;
  unsigned char* a_lo = smem + a_bytes;
  unsigned char* b_hi = smem + (SPLIT == 3 ? 2 : 1) * a_bytes;
  unsigned char* b_lo = b_hi + b_bytes;
  unsigned char* tail = b_hi + (SPLIT == 3 ? 2 : 1) * b_bytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tail);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tail + 8);
  int* tgt = reinterpret_cast<int*>(tail + 16);          // [NW]
  int* unfold = reinterpret_cast<int*>(tail + 16 + 4 * NW);  // [Kp] -> r*n+s, or -1
  int* wait_ok = reinterpret_cast<int*>(tail + 12);
  // epilogue staging [16][kTileM] reuses the A tile, which the completed MMA no longer reads
  float* stage = reinterpret_cast<float*>(a_hi);
  float* crow_s = reinterpret_cast<float*>(tail + 16 + 4 * NW + 4 * Kp);  // [Nb] when A.crow_smem

  const int64_t Ja = blockIdx.x;
  const int64_t a_beg = A.a_srow[Ja], a_end = A.a_srow[Ja + 1];
  if (a_beg == a_end) return;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int k = tid; k < Kp; k += kThreads) {
    int v = -1;
    if (k < A.K) {
      int r = 0;
      while ((r + 1) * (r + 2) / 2 <= k) ++r;
      v = r * n + (k - r * (r + 1) / 2);
    }
    unfold[k] = v;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(NW));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = make_idesc(kTileM, NW);
  const float* crow = A.C + Ja * A.Nb;
  if (A.crow_smem) {
    for (int64_t j = tid; j < A.Nb; j += kThreads) crow_s[j] = crow[j];
    crow = crow_s;
  }
  uint32_t phase = 0;
  bool ok = true;
  __syncthreads();

  for (int64_t a0 = a_beg; a0 < a_end && ok; a0 += NW) {
    const int cnt = (int)min64(NW, a_end - a0);
    // B operand: rows a = alpha singles of Ja, columns k = folded rs
    for (int i0 = tid; i0 < NW * Kp; i0 += 8 * kThreads) {
      // eight integral values in flight before any shared-memory store
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + u * kThreads;
        v[u] = 0.0f;
        if (i < NW * Kp) {
          const int a = i / Kp, k = i - a * Kp;
          const int rs = unfold[k];
          if (a < cnt && rs >= 0) {
            const int sp = __ldg(&A.a_slink[a0 + a].y);
            const int pq = (sp > 0 ? sp : -sp) - 1;
            v[u] = __ldg(A.eri + (int64_t)pq * n2 + rs);
            if (sp < 0) v[u] = -v[u];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + u * kThreads;
        if (i >= NW * Kp) break;
        const int a = i / Kp, k = i - a * Kp;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v[u]);
        *reinterpret_cast<__nv_bfloat16*>(b_hi + tile_off(a, k, KB)) = hi;
        if (SPLIT == 3)
          *reinterpret_cast<__nv_bfloat16*>(b_lo + tile_off(a, k, KB)) =
              __float2bfloat16_rn(v[u] - __bfloat162float(hi));
      }
    }
    if (tid < NW) tgt[tid] = (tid < cnt) ? A.a_slink[a0 + tid].x : 0;

    for (int64_t ib0 = 0; ib0 < A.Nb && ok; ib0 += kTileM) {
      // A operand: row m = beta string ib0 + m, zero then scatter D entries
      const int m = tid;
      const int64_t Ib = ib0 + m;
      for (int kb = 0; kb < KB; ++kb) {
        *reinterpret_cast<uint4*>(a_hi + tile_off(m, kb * 8, KB)) = make_uint4(0, 0, 0, 0);
        if (SPLIT == 3)
          *reinterpret_cast<uint4*>(a_lo + tile_off(m, kb * 8, KB)) = make_uint4(0, 0, 0, 0);
      }
      if (Ib < A.Nb) {
        const int nk = __ldg(A.b_cnt + Ib);
        const int2* __restrict__ ell = A.b_ell + Ib;
        for (int k0 = 0; k0 < nk; k0 += 8) {
          // eight link records in flight before any shared-memory store
          int2 l[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            l[u] = (k0 + u < nk) ? __ldg(ell + (int64_t)(k0 + u) * A.Nb) : make_int2(0, 0);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (k0 + u >= nk) break;
            const int pair = (l[u].y > 0 ? l[u].y : -l[u].y) - 1;
            float v = crow[l[u].x];
            if (l[u].y < 0) v = -v;
            const int kf = fold_index(pair / n, pair % n);
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            *reinterpret_cast<__nv_bfloat16*>(a_hi + tile_off(m, kf, KB)) = hi;
            if (SPLIT == 3)
              *reinterpret_cast<__nv_bfloat16*>(a_lo + tile_off(m, kf, KB)) =
                  __float2bfloat16_rn(v - __bfloat162float(hi));
          }
        }
      }
      fence_proxy_async();
      fence_before();
      __syncthreads();
      fence_after();
      if (tid == 0) {
        const uint32_t sbo_a = (uint32_t)KB * 128, sbo_b = (uint32_t)KB * 128;
        const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi),
                       bl = smem_u32(b_lo);
        uint32_t acc = 0;
        for (int kk = 0; kk < KB / 2; ++kk) {
          const uint32_t off = (uint32_t)kk * 256;  // 16 K-elements = two core matrices
          mma_bf16(tmem, make_desc(ah + off, 128, sbo_a), make_desc(bh + off, 128, sbo_b), idesc,
                   acc);
          acc = 1;
          if (SPLIT == 3) {
            mma_bf16(tmem, make_desc(ah + off, 128, sbo_a), make_desc(bl + off, 128, sbo_b),
                     idesc, 1);
            mma_bf16(tmem, make_desc(al + off, 128, sbo_a), make_desc(bh + off, 128, sbo_b),
                     idesc, 1);
          }
        }
        mma_commit(smem_u32(mbar));
        // one thread polls the barrier (bounded) and tells the block
        bool done = mbar_wait(smem_u32(mbar), phase);
        if (!done) {
          atomicExch(&g_tc_error, 1);
          // a second bounded chance for the MMAs in flight before TMEM is freed
          mbar_wait(smem_u32(mbar), phase);
        }
        *wait_ok = done ? 1 : 0;
      }
      __syncthreads();
      if (!*wait_ok) {
        ok = false;
        break;
      }
      phase ^= 1u;
      fence_after();
      // epilogue: row m of E lives in TMEM lane m; warp w reads lanes 32w..32w+31
      const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
#pragma unroll 1
      for (int c0 = 0; c0 < NW && c0 < cnt; c0 += 16) {
        float e[16];
        tmem_ld16(tmem + lane_base + (uint32_t)c0, e);
#pragma unroll
        for (int i = 0; i < 16; ++i) stage[i * kTileM + m] = e[i];
        __syncthreads();
        // transpose through shared memory: each thread adds four consecutive beta
        // strings of one target row at a time (vector atomics, 4x fewer operations)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int idx = tid + j * kThreads;  // 0..511
          const int ci = idx >> 5, m4 = (idx & 31) * 4;
          const int a = c0 + ci;
          const int64_t ib = ib0 + m4;
          if (a < cnt && ib < A.Nb) {
            float* dst = A.sig + (int64_t)tgt[a] * A.Nb + ib;
            const float* src = stage + ci * kTileM + m4;
            if (A.vec4 && ib + 3 < A.Nb) {
              atomicAdd(reinterpret_cast<float4*>(dst), make_float4(src[0], src[1], src[2], src[3]));
            } else {
              for (int q = 0; q < 4 && ib + q < A.Nb; ++q) atomicAdd(dst + q, src[q]);
            }
          }
        }
        __syncthreads();
      }
      fence_before();
      __syncthreads();
      fence_after();
    }
    __syncthreads();
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NW));
  }
}

template <int NW, int SPLIT>
static int launch(const Args& a, cudaStream_t s) {
  const int Kp = a.KB * 8;
  const size_t a_region = std::max<size_t>((size_t)kTileM * Kp * 2, 16 * kTileM * 4);
  size_t bytes = (size_t)(SPLIT == 3 ? 2 : 1) * (a_region + (size_t)NW * Kp * 2) + 16 + 4 * NW +
                 4 * Kp + 64;
  Args b = a;
  b.crow_smem = (bytes + 4 * a.Nb <= 200 * 1024) ? 1 : 0;
  if (b.crow_smem) bytes += 4 * a.Nb;
  if (bytes > 220 * 1024)
    return fail(HINQS_ERR_ARG, "tensor-core sigma: tile of %zu bytes exceeds shared memory (n_orb=%d)",
                bytes, a.n);
  auto kern = k_sigma_ab_tc<NW, SPLIT>;
  HQ_TRY(allow_max_smem(kern));
  kern<<<(unsigned)a.Na, kThreads, bytes, s>>>(b);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

}  // namespace tc

int sigma_ab_tc_launch(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                       const hinqs_links_s* lb, const float* c, float* sig, int split,
                       cudaStream_t s) {
  tc::Args a;
  a.Na = B->Na;
  a.Nb = B->Nb;
  a.n = H->n;
  a.K = H->n * (H->n + 1) / 2;
  a.KB = (int)ceil_div(a.K, 16) * 2;
  a.a_srow = la->srow_ptr;
  a.a_slink = la->slink;
  a.b_ell = lb->sell;
  a.b_cnt = lb->scount;
  a.eri = H->eri32;
  a.C = c;
  a.sig = sig;
  a.crow_smem = 0;
  a.vec4 = (B->Nb % 4 == 0) ? 1 : 0;
  const bool wide = la->max_srow > 64;
  if (split == 3) return wide ? tc::launch<128, 3>(a, s) : tc::launch<64, 3>(a, s);
  return wide ? tc::launch<128, 1>(a, s) : tc::launch<64, 1>(a, s);
}

int tc_error_check(cudaStream_t s) {
  int h = 0;
  HQ_CUDA(cudaMemcpyFromSymbolAsync(&h, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  HQ_CUDA(cudaStreamSynchronize(s));
  if (h) {
    int z = 0;
    cudaMemcpyToSymbolAsync(g_tc_error, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    return fail(HINQS_ERR_TIMEOUT, "tensor-core sigma: a bounded wait on the MMA barrier ran out");
  }
  return HINQS_OK;
}

}  // namespace hinqs
