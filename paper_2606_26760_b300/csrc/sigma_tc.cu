// K5 -> K6 -> K7 on the 5th-generation tensor cores: the opposite-spin part of
// sigma written as a gather into D followed by a dense GEMM against (pq|rs),
//
//   sigma(Ia,Ib) += sum_{alpha singles Ja -> Ia, pair pq, sign s_a} s_a E(Ja,Ib;pq),
//   E(Ja,Ib;pq)   = sum_rs (pq|rs) D(Ja,Ib;rs),
//   D(Ja,Ib;rs)   = sum_{beta singles Ib -> Jb with pair rs} s_b C(Ja,Jb)
//                   + [rs = jj, j in Ib] C(Ja,Ib).
//
// Work unit: one alpha string Ja and a chunk of at most NW of its alpha singles.
// The (pq|.) rows of those singles form the B operand [NW x K], copied from a
// BF16 table prepared with the Hamiltonian (the sign of the single flips the BF16
// sign bits); each tile of 128 beta strings forms the A operand D [128 x K],
// gathered from the row C(Ja, :).  Both are BF16 in shared memory (K-major,
// canonical no-swizzle layout of 8x16-byte core matrices); K runs over the folded
// pairs r >= s (the integral is symmetric in r,s and a beta string contributes at
// most one of rs, sr), padded to a multiple of 16.  One thread issues the
// tcgen05.mma chain into an FP32 accumulator in tensor memory.  With two stages the
// gather of tile t+1 overlaps the MMA of tile t, each stage with its own A buffer,
// tensor-memory columns and mbarrier.  The accumulator is read back with tcgen05.ld
// (lane = beta string) and added into sigma with coalesced reductions.  CTAs are
// persistent (at most what shared and tensor memory hold per SM) and stride over
// the alpha strings.  SPLIT = 3 represents each operand as hi + lo BF16 terms and
// accumulates hi*hi + hi*lo + lo*hi (about 16 significant bits); SPLIT = 1 uses hi.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "hinqs_internal.cuh"

namespace hinqs {

__device__ int g_tc_error = 0;  // set by a CTA whose bounded wait ran out

namespace tc {

constexpr int kThreads = 256;
constexpr int kTileM = 128;
// packed slot quads a gather thread has in flight (measured on B300: six, or an L1
// prefetch of the next tile's quads during the MMA, gain nothing)
constexpr int kQuads = 4;
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

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase,
                                          long long limit = kWaitLimit) {
  for (long long it = 0; it < limit; ++it) {
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
  int n, KB;  // KB = padded folded K / 8 (16-byte chunks per operand row)
  const int64_t* a_srow;
  const int2* a_slink;
  const int2* b_ell;  // pair-major {Jb, kpart | sign bit} (tensor-core gather slots)
  const uint4* b_q;   // the same slots packed, quad-major (null: use b_ell)
  int wq;             // quads per row of b_q
  const int* b_cnt;
  const uint4* Bhi;  // [n*n][KB] BF16 rows of (pq|.) over the folded pairs
  const uint4* Blo;  // low parts (SPLIT = 3)
  const float* C;
  float* sig;
  int crow_smem;  // stage the row C(Ja, :) in shared memory
};

// A device work queue of (problem, alpha string) items for the batched launch: problem
// r has starts[r+1] - starts[r] alpha strings (starts[0] = 0, starts[R] = total), and
// CTAs take items in turn from *counter.  reqs == NULL: one problem, the kernel's Args.
struct Queue {
  const Args* reqs = nullptr;
  const int64_t* starts = nullptr;
  int R = 0;
  unsigned long long* counter = nullptr;
  int64_t total = 0;
};

// The problems of one batched launch, passed by value as a kernel parameter (no host to
// device copy, so that a launch never waits for the host): kMaxBatch problems at most
// per launch, a longer batch is split.
constexpr int kMaxBatch = 48;
struct BatchTab {
  Args reqs[kMaxBatch];
  int64_t starts[kMaxBatch + 1];
  int R;
  int64_t total;
};

// Shared-memory bytes of one CTA (the layout of the kernel below).
__host__ __device__ inline size_t smem_bytes(int NW, int SPLIT, int STAGES, int KB, int64_t Nb,
                                             bool crow) {
  const size_t np = SPLIT == 3 ? 2 : 1;
  size_t x = STAGES * np * (size_t)kTileM * KB * 16 + np * (size_t)NW * KB * 16 + 32 + 8 * NW;
  x = (x + 15) & ~(size_t)15;
  if (crow) x += (SPLIT == 1 ? 2 : 4) * (size_t)Nb;  // the row as BF16 (SPLIT 1) or FP32
  return x;
}

// Persistent CTAs of 8 warps; each takes alpha strings Ja = blockIdx.x, +gridDim.x, ...
// (or, in the batched launch, (problem, alpha string) items from the work queue) and,
// per chunk of at most NW alpha singles of Ja, runs the beta tiles through a
// STAGES-deep pipeline: while the MMA of tile t runs, the warps gather D for tile
// t+1 into the other A buffer; then they read tile t's accumulator (its own TMEM
// columns) and add it into sigma with coalesced reductions (lane = beta string).
template <int NW, int SPLIT, int STAGES>
__device__ __forceinline__ void sigma_ab_tc_body(const Args& A0, const Queue& Q) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ int64_t s_item;
  __shared__ int s_req;
  constexpr int NP = SPLIT == 3 ? 2 : 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  Args A = A0;
  const int KB = A.KB;  // the same for every problem of a batch
  int64_t Nb = A.Nb;
  const uint32_t a_bytes = (uint32_t)kTileM * KB * 16;
  const uint32_t b_bytes = (uint32_t)NW * KB * 16;
  unsigned char* a_buf = smem;                              // [STAGES][NP][a_bytes]
  unsigned char* b_buf = smem + STAGES * NP * a_bytes;      // [NP][b_bytes]
  unsigned char* tail = b_buf + NP * b_bytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tail);       // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tail + 16);
  int* wait_flag = reinterpret_cast<int*>(tail + 20);
  float** tgt = reinterpret_cast<float**>(tail + 32);       // [NW] target rows of sigma
  float* crow_s = reinterpret_cast<float*>(
      smem + ((STAGES * NP * a_bytes + NP * b_bytes + 32 + 8 * NW + 15) & ~15u));

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar + 1)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(STAGES * NW));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = make_idesc(kTileM, NW);
  const uint32_t sbo = (uint32_t)KB * 128;
  uint32_t ph0 = 0, ph1 = 0;
  bool ok = true;
  int T = (int)((Nb + kTileM - 1) / kTileM);

  // zero one A stage (both planes)
  auto zero_stage = [&](int st) {
    uint4* z = reinterpret_cast<uint4*>(a_buf + (size_t)st * NP * a_bytes);
    const int cnt16 = (int)(NP * a_bytes / 16);
    for (int i = tid; i < cnt16; i += kThreads) z[i] = make_uint4(0, 0, 0, 0);
  };
  // gather D for beta tile t into stage st: row m = beta string, two threads per row
  auto build_d = [&](int t, int st, const float* crow) {
    const int m = tid & (kTileM - 1), hh = tid >> 7;
    unsigned char* ah = a_buf + (size_t)st * NP * a_bytes + (m >> 3) * (KB * 128) + (m & 7) * 16;
    const int64_t Ib = (int64_t)t * kTileM + m;
    // D(Ib, kf) = sign * C(Ja, Jb) at byte offset off of the row; with one BF16 term and
    // the row staged, the row is BF16 already (BF16 rounding commutes with the sign)
    auto put16 = [&](uint32_t jb, uint32_t off, uint32_t neg) {
      const unsigned short b = reinterpret_cast<const unsigned short*>(crow)[jb];
      *reinterpret_cast<unsigned short*>(ah + off) = b ^ (unsigned short)(neg >> 16);
    };
    auto put32 = [&](uint32_t jb, uint32_t off, uint32_t neg) {
      const float v = __uint_as_float(__float_as_uint(crow[jb]) ^ neg);
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      *reinterpret_cast<__nv_bfloat16*>(ah + off) = hi;
      if (SPLIT == 3)
        *reinterpret_cast<__nv_bfloat16*>(ah + a_bytes + off) =
            __float2bfloat16_rn(v - __bfloat162float(hi));
    };
    auto gather = [&](auto put) {
      const int nk = __ldg(A.b_cnt + Ib);
      if (A.b_q) {
        // packed quad-major slots: thread hh takes quads hh, hh + 2, ...; four quads
        // (sixteen records) in flight, the first four loaded without waiting for nk
        // (every quad below wq exists, zero-padded)
        const uint4* __restrict__ q4 = A.b_q + Ib;
        for (int j0 = hh; j0 < A.wq && (j0 == hh || 4 * j0 < nk); j0 += 2 * kQuads) {
          uint4 l[kQuads];
#pragma unroll
          for (int u = 0; u < kQuads; ++u)
            l[u] = (j0 + 2 * u < A.wq) ? __ldg(q4 + (int64_t)(j0 + 2 * u) * Nb)
                                       : make_uint4(0, 0, 0, 0);
#pragma unroll
          for (int u = 0; u < 4 * kQuads; ++u) {
            const int k = 4 * (j0 + 2 * (u >> 2)) + (u & 3);
            if (k >= nk) break;
            const uint4 q = l[u >> 2];
            const uint32_t y = (u & 3) == 0 ? q.x : (u & 3) == 1 ? q.y : (u & 3) == 2 ? q.z : q.w;
            put(y & 0x1ffffu, (y >> 17) & 0x3fffu, y & 0x80000000u);
          }
        }
      } else {
        // pair-major slots: thread hh takes slot pairs hh, hh + 2, ...; one 16-byte load
        // per pair, four pairs (eight records) in flight before any shared-memory store
        const int4* __restrict__ ell = reinterpret_cast<const int4*>(A.b_ell) + Ib;
        const int np = (nk + 1) >> 1;
        for (int j0 = hh; j0 < np; j0 += 8) {
          int4 l[4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            l[u] = (j0 + 2 * u < np) ? __ldg(ell + (int64_t)(j0 + 2 * u) * Nb)
                                     : make_int4(0, 0, 0, 0);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int k = 2 * (j0 + 2 * (u >> 1)) + (u & 1);
            if (k >= nk) break;
            const int x = (u & 1) ? l[u >> 1].z : l[u >> 1].x;
            const uint32_t y = (uint32_t)((u & 1) ? l[u >> 1].w : l[u >> 1].y);
            put((uint32_t)x, y & 0x7fffffffu, y & 0x80000000u);
          }
        }
      }
    };
    if (Ib < Nb) {
      if (SPLIT == 1 && A.crow_smem) gather(put16);
      else gather(put32);
    }
    fence_proxy_async();  // generic-proxy writes (zeroing and gather) -> tensor-core reads
  };
  // one thread issues the MMA chain of stage st and commits it to mbar[st]
  auto issue = [&](int st) {
    const uint32_t ah = smem_u32(a_buf + (size_t)st * NP * a_bytes), al = ah + a_bytes;
    const uint32_t bh = smem_u32(b_buf), bl = bh + b_bytes;
    const uint32_t d = tmem + (uint32_t)(st * NW);
    for (int kk = 0; kk < KB / 2; ++kk) {
      const uint32_t off = (uint32_t)kk * 256;  // 16 K-elements = two core matrices
      mma_bf16(d, make_desc(ah + off, 128, sbo), make_desc(bh + off, 128, sbo), idesc,
               kk > 0 ? 1u : 0u);
      if (SPLIT == 3) {
        mma_bf16(d, make_desc(ah + off, 128, sbo), make_desc(bl + off, 128, sbo), idesc, 1u);
        mma_bf16(d, make_desc(al + off, 128, sbo), make_desc(bh + off, 128, sbo), idesc, 1u);
      }
    }
    mma_commit(smem_u32(mbar + st));
  };

  int64_t next_ja = blockIdx.x;
  for (;;) {
    int64_t Ja;
    if (Q.reqs) {
      __syncthreads();  // the previous item's readers of A, crow_s, b_buf and tgt are done
      if (tid == 0) {
        const int64_t item = (int64_t)atomicAdd(Q.counter, 1ull);
        int r = 0;
        if (item < Q.total) {  // the problem whose range holds the item
          int lo = 0, hi = Q.R;
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (Q.starts[mid] <= item) lo = mid;
            else hi = mid;
          }
          r = lo;
        }
        s_item = item;
        s_req = r;
      }
      __syncthreads();
      if (s_item >= Q.total || !ok) break;
      A = Q.reqs[s_req];
      Ja = s_item - Q.starts[s_req];
      Nb = A.Nb;
      T = (int)((Nb + kTileM - 1) / kTileM);
    } else {
      if (next_ja >= A.Na || !ok) break;
      Ja = next_ja;
      next_ja += gridDim.x;
    }
    const int64_t a_beg = A.a_srow[Ja], a_end = A.a_srow[Ja + 1];
    if (a_beg == a_end) continue;
    const float* crow = A.C + Ja * Nb;
    __syncthreads();  // the previous string's readers of crow_s, b_buf and tgt are done
    if (A.crow_smem) {
      if (SPLIT == 1) {
        unsigned short* c16 = reinterpret_cast<unsigned short*>(crow_s);
        for (int64_t j = tid; j < Nb; j += kThreads)
          c16[j] = __bfloat16_as_ushort(__float2bfloat16_rn(crow[j]));
      } else {
        for (int64_t j = tid; j < Nb; j += kThreads) crow_s[j] = crow[j];
      }
      crow = crow_s;
    }
    for (int64_t a0 = a_beg; a0 < a_end && ok; a0 += NW) {
      const int cnt = (int)min64(NW, a_end - a0);
      // B operand: the (pq|.) rows of the alpha singles, sign folded into the BF16 sign bits
      for (int i = tid; i < NW * KB; i += kThreads) {
        const int a = i / KB, kb = i - a * KB;
        uint4 vh = make_uint4(0, 0, 0, 0), vl = make_uint4(0, 0, 0, 0);
        if (a < cnt) {
          const int sp = __ldg(&A.a_slink[a0 + a].y);
          const int64_t row = (int64_t)((sp > 0 ? sp : -sp) - 1) * KB + kb;
          vh = __ldg(A.Bhi + row);
          if (SPLIT == 3) vl = __ldg(A.Blo + row);
          if (sp < 0) {
            vh.x ^= 0x80008000u, vh.y ^= 0x80008000u, vh.z ^= 0x80008000u, vh.w ^= 0x80008000u;
            vl.x ^= 0x80008000u, vl.y ^= 0x80008000u, vl.z ^= 0x80008000u, vl.w ^= 0x80008000u;
          }
        }
        *reinterpret_cast<uint4*>(b_buf + tile_off(a, kb * 8, KB)) = vh;
        if (SPLIT == 3) *reinterpret_cast<uint4*>(b_buf + b_bytes + tile_off(a, kb * 8, KB)) = vl;
      }
      if (tid < NW) tgt[tid] = A.sig + (tid < cnt ? (int64_t)A.a_slink[a0 + tid].x * Nb : 0);
      for (int st = 0; st < STAGES; ++st) zero_stage(st);
      __syncthreads();
      build_d(0, 0, crow);
      fence_before();
      __syncthreads();
      fence_after();
      if (tid == 0) issue(0);

      for (int t = 0; t < T; ++t) {
        const int st = STAGES == 2 ? (t & 1) : 0;
        if (STAGES == 2 && t + 1 < T) {
          build_d(t + 1, st ^ 1, crow);  // overlaps the MMA of tile t
          fence_before();
          __syncthreads();
          fence_after();
          if (tid == 0) issue(st ^ 1);
        }
        // one thread waits (bounded) for tile t's MMA chain and tells the block, so
        // that the other warps sleep at the barrier instead of spinning on the
        // mbarrier (their issue slots go to the other resident CTAs)
        if (tid == 0) *wait_flag = mbar_wait(smem_u32(mbar + st), st == 0 ? ph0 : ph1) ? 1 : 0;
        __syncthreads();
        const bool done = *wait_flag != 0;
        if (st == 0) ph0 ^= 1u;
        else ph1 ^= 1u;
        if (done) {
          fence_after();
          // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (beta strings) and the
          // 16-column groups of its half; lane = beta string, so each reduction of one
          // alpha target row is a coalesced 128-byte access
          const int q = warp & 3;
          const int64_t ib = (int64_t)t * kTileM + 32 * q + lane;
          const uint32_t lane_base = (uint32_t)(32 * q) << 16;
#pragma unroll 1
          for (int c0 = 16 * (warp >> 2); c0 < cnt; c0 += 32) {
            float e[16];
            tmem_ld16(tmem + lane_base + (uint32_t)(st * NW + c0), e);
            if (ib < Nb) {
#pragma unroll
              for (int i = 0; i < 16; ++i)
                if (c0 + i < cnt) atomicAdd(tgt[c0 + i] + ib, e[i]);
            }
          }
          zero_stage(st);  // ready for the gather of tile t + STAGES
        }
        fence_before();
        if (__syncthreads_or(done ? 0 : 1)) {
          ok = false;
          if (tid == 0) {
            atomicExch(&g_tc_error, 1);
            // a second bounded chance for the MMAs in flight before TMEM is freed
            mbar_wait(smem_u32(mbar + st), st == 0 ? ph0 ^ 1u : ph1 ^ 1u);
            if (STAGES == 2 && t + 1 < T)
              mbar_wait(smem_u32(mbar + (st ^ 1)), st == 0 ? ph1 : ph0);
          }
          __syncthreads();
          break;
        }
        fence_after();
        if (STAGES == 1 && t + 1 < T) {
          build_d(t + 1, 0, crow);
          fence_before();
          __syncthreads();
          fence_after();
          if (tid == 0) issue(0);
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(STAGES * NW));
  }
}

// One stage of at most 64 columns is meant to run three CTAs per SM: the register cap
// keeps them there (80 a thread).
template <int NW, int SPLIT, int STAGES>
__global__ void __launch_bounds__(kThreads) __maxnreg__((NW <= 64 && STAGES == 1) ? 80 : 128) k_sigma_ab_tc(Args A) {
  sigma_ab_tc_body<NW, SPLIT, STAGES>(A, Queue{});
}

// The batched form: the table lives in the parameter space for the whole launch.
template <int NW, int SPLIT, int STAGES>
__global__ void __launch_bounds__(kThreads, (NW <= 64 && STAGES == 1) ? 3 : 1) k_sigma_ab_tc_batch(
    const __grid_constant__ BatchTab tab, unsigned long long* counter) {
  Queue q;
  q.reqs = tab.reqs;
  q.starts = tab.starts;
  q.R = tab.R;
  q.counter = counter;
  q.total = tab.total;
  sigma_ab_tc_body<NW, SPLIT, STAGES>(tab.reqs[0], q);
}

// BF16 (hi, lo) rows of the folded integral matrix: row pq, column k < K holds
// (pq|rs) for the k-th folded pair (r >= s), columns K..8KB-1 are zero.
__global__ void k_btable(const float* __restrict__ eri32, int n, int K, int KB,
                         __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int n2 = n * n, Kp = KB * 8;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n2 * Kp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int pq = (int)(i / Kp), k = (int)(i % Kp);
    float v = 0.0f;
    if (k < K) {
      int r = 0;
      while ((r + 1) * (r + 2) / 2 <= k) ++r;
      v = eri32[(int64_t)pq * n2 + r * n + (k - r * (r + 1) / 2)];
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// Resident CTAs per SM of k_sigma_ab_tc<NW, SPLIT, STAGES> with a CTA of `bytes` of
// shared memory: as many as shared memory, registers and threads allow, but never more
// than the 512 tensor-memory columns hold; *req is the shared-memory request that
// keeps the scheduler there (padding it, so that no CTA waits in tcgen05.alloc for
// another to finish).  228 KB of shared memory per SM, 1 KB reserved per CTA.
template <int NW, int SPLIT, int STAGES>
static int ctas_per_sm(size_t bytes, size_t* req) {
  auto kern = k_sigma_ab_tc<NW, SPLIT, STAGES>;
  const int cap = 512 / (STAGES * NW);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;
  const int by_regs = 65536 / (warp_regs * (kThreads / 32));
  const int by_threads = 2048 / kThreads;
  size_t r = bytes;
  if ((int)(233472 / (r + 1024)) > cap) r = 233472 / (cap + 1);  // 1 KB margin
  if (req) *req = r;
  return std::min(std::min(cap, (int)(233472 / (r + 1024))), std::min(by_regs, by_threads));
}

template <int NW, int SPLIT, int STAGES>
static int launch(const Args& a, bool crow, cudaStream_t s) {
  Args b = a;
  b.crow_smem = crow ? 1 : 0;
  const size_t bytes = smem_bytes(NW, SPLIT, STAGES, a.KB, a.Nb, crow);
  auto kern = k_sigma_ab_tc<NW, SPLIT, STAGES>;
  HQ_TRY(allow_max_smem(kern));
  size_t req = bytes;
  const int per_sm = ctas_per_sm<NW, SPLIT, STAGES>(bytes, &req);
  if (per_sm < 1)
    return fail(HINQS_ERR_ARG, "tensor-core sigma: a CTA of %zu bytes does not fit an SM", bytes);
  const int grid = (int)std::min<int64_t>(a.Na, (int64_t)per_sm * kNumSMs);
  kern<<<grid, kThreads, req, s>>>(b);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

// The batched launch: one persistent grid over the (problem, alpha string) items of
// every problem in reqs (same n_orb; the C row staged when the largest fits), one
// stage, kMaxBatch problems per launch.  kTcNoFit when the operand tiles do not fit.
// Nothing waits for the device: the table is a kernel parameter and the item counter
// a stream-ordered allocation.
template <int NW, int SPLIT>
static int launch_batch(std::vector<Args>& reqs, cudaStream_t s) {
  int64_t nb_max = 0;
  for (const Args& a : reqs) nb_max = std::max(nb_max, a.Nb);
  const size_t lim = (size_t)smem_optin_limit();
  const int KB = reqs[0].KB;
  const bool crow = smem_bytes(NW, SPLIT, 1, KB, nb_max, true) <= lim;
  if (!crow && smem_bytes(NW, SPLIT, 1, KB, nb_max, false) > lim) return kTcNoFit;
  const size_t bytes = smem_bytes(NW, SPLIT, 1, KB, nb_max, crow);
  auto kern = k_sigma_ab_tc_batch<NW, SPLIT, 1>;
  HQ_TRY(allow_max_smem(kern));
  const int cap = 512 / NW;
  cudaFuncAttributes fa;
  HQ_CUDA(cudaFuncGetAttributes(&fa, kern));
  const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;
  const int by_regs = 65536 / (warp_regs * (kThreads / 32));
  size_t req = bytes;
  if ((int)(233472 / (req + 1024)) > cap) req = 233472 / (cap + 1);
  const int per_sm = std::min(std::min(cap, (int)(233472 / (req + 1024))),
                              std::min(by_regs, 2048 / kThreads));
  if (per_sm < 1) return kTcNoFit;
  const int chunks = (int)((reqs.size() + kMaxBatch - 1) / kMaxBatch);
  unsigned long long* d_counter = nullptr;
  HQ_TRY(dalloc(&d_counter, (size_t)chunks, s));
  auto run = [&]() -> int {
    HQ_CUDA(cudaMemsetAsync(d_counter, 0, chunks * sizeof(unsigned long long), s));
    for (int c = 0; c < chunks; ++c) {
      BatchTab tab;
      const size_t r0 = (size_t)c * kMaxBatch;
      tab.R = (int)std::min<size_t>(kMaxBatch, reqs.size() - r0);
      tab.starts[0] = 0;
      for (int r = 0; r < tab.R; ++r) {
        tab.reqs[r] = reqs[r0 + r];
        tab.reqs[r].crow_smem = crow ? 1 : 0;
        tab.starts[r + 1] = tab.starts[r] + tab.reqs[r].Na;
      }
      tab.total = tab.starts[tab.R];
      if (tab.total == 0) continue;
      const int grid = (int)std::min<int64_t>(tab.total, (int64_t)per_sm * kNumSMs);
      kern<<<grid, kThreads, req, s>>>(tab, d_counter + c);
      HQ_LAUNCH_CHECK();
    }
    return HINQS_OK;
  };
  const int rc = run();
  dfree(d_counter, s);
  return rc;
}

// Largest configuration that fits: two stages with the C row in shared memory, then
// without the row, then one stage (stages = 1: one stage only, which leaves room for
// more resident CTAs per SM).
template <int NW, int SPLIT>
static int launch_fit(const Args& a, int stages, cudaStream_t s) {
  const size_t lim = (size_t)smem_optin_limit();
  if (stages != 1) {
    if (smem_bytes(NW, SPLIT, 2, a.KB, a.Nb, true) <= lim) return launch<NW, SPLIT, 2>(a, true, s);
    if (smem_bytes(NW, SPLIT, 2, a.KB, a.Nb, false) <= lim) return launch<NW, SPLIT, 2>(a, false, s);
  }
  // one stage, the C row in shared memory when it fits (measured on B300: four CTAs of
  // 64 registers reading the row through L1 run slower than three that stage it)
  if (smem_bytes(NW, SPLIT, 1, a.KB, a.Nb, true) <= lim) return launch<NW, SPLIT, 1>(a, true, s);
  if (smem_bytes(NW, SPLIT, 1, a.KB, a.Nb, false) <= lim) return launch<NW, SPLIT, 1>(a, false, s);
  return kTcNoFit;
}

template <int NW, int SPLIT>
static bool fits(const Args& a) {
  return smem_bytes(NW, SPLIT, 1, a.KB, a.Nb, false) <= (size_t)smem_optin_limit();
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Tile-stationary, warp-specialised form of the same term (BF16 operands, n <= 22,
// at most 64 alpha singles per string, at most 64 gather slots per beta string).
//
// A CTA works through items (beta tile t, alpha string Ja), tile by tile, so that a
// beta tile's gather slots and the non-zero pattern of D stay fixed while the alpha
// strings change: each gather thread keeps its slots in registers for the whole tile,
// and a D stage is cleared only when it meets a new tile (every item of a tile writes
// the same positions).  The whole folded table (pq|rs) stays in shared memory for the
// CTA's life; per item, the rows of Ja's singles (signs folded into the BF16 sign
// bits) are copied from it into a B stage of N = 16..64 rows, so that the accumulator
// holds exactly the singles' columns and the epilogue reads them 16 columns at a time.
// Warp roles, with mbarrier handoffs and no block-wide barrier inside the loop:
//   warp 0      copies the row C(Ja, :) into a shared stage (one cp.async.bulk when
//               the rows are 16-byte aligned, else plain loads)
//   warp 1      one thread issues the tcgen05.mma chain of each item (K = Kp in
//               steps of 16) into one of two tensor-memory accumulators
//   warps 2-9   gather: two threads per beta string (its even and odd slots) write D
//               into one of two shared stages; the warps also copy the item's B rows
//   warps 10-13 epilogue: tcgen05.ld of the accumulator (lane = beta string) and
//               reductions into sigma (a warp covers 32 consecutive beta strings of one
//               target row)
// Items of CTA b: the alpha strings Ja = b, b + G, b + 2G, ... (G CTAs) for every
// beta tile, tiles visited from tile b mod T on; each role walks them with counters
// (no integer division in the loop).  Every wait is bounded and suspends the waiting
// thread; when one gives up the CTA raises the error flag, the other roles stop at
// their next wait or item, and the copies and MMAs in flight are waited for (bounded)
// before tensor memory is freed.
namespace tc2 {

using tc::fence_after;
using tc::fence_before;
using tc::fence_proxy_async;
using tc::make_desc;
using tc::make_idesc;
using tc::mma_bf16;
using tc::mma_commit;
using tc::smem_u32;

constexpr int kWarps = 14;
constexpr int kThreads = 32 * kWarps;
constexpr int kTileM = 128;
constexpr int kMaxKp = 256;        // folded K of the stationary table (n <= 22)
constexpr int kMaxSingles = 64;    // N of one item's MMA (alpha singles of one string)
constexpr int kMaxSlots = 64;      // gather slots (beta singles + occupied) per beta string
constexpr int kThreadsPerRow = 2;  // gather threads of one beta string
constexpr int kMySlots = kMaxSlots / kThreadsPerRow;
constexpr int kTmemCols = 128;     // two accumulators of kMaxSingles columns
constexpr int kGatherWarps = 8;
constexpr int kGather = 32 * kGatherWarps;
constexpr int kEpiWarps = 4;
constexpr int kSlotJbBits = 19;    // packed slot: Jb | kpart << 19 | sign << 31
// A waiting thread polls with a growing sleep between polls (16 to 256 ns) and gives
// up after kWaitNs of wall time (the global timer): a legitimate wait here lasts
// microseconds, also on a GPU shared with other work.
constexpr uint32_t kSuspendNs = 20000;
constexpr uint64_t kWaitNs = 2000000000ull;

struct Args {
  int64_t Na, Nb, T;
  int n, KB, Kp;
  const int64_t* a_srow;
  const int2* a_slink;
  const int2* b_tcell;  // pair-major {Jb, kpart | sign << 31}
  const int* b_cnt;
  const uint4* Bimg;    // shared-memory image of the folded table, Kp * KB chunks
  const float* C;
  float* sig;
  int bulk_row;         // rows of C may be fetched with one cp.async.bulk
  uint32_t off_Bs, off_D, off_C, off_F, off_bar, crow_stride;
};

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b))
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_u32(b)),
               "r"(bytes)
               : "memory");
}
// bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from global
// memory into shared memory, completing on the mbarrier's transaction count
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(b))
      : "memory");
}
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool wait_phase(uint64_t* b, uint32_t parity) {
  const uint32_t a = smem_u32(b);
  const uint64_t t0 = global_ns();
  uint32_t sleep_ns = 16;
  for (uint32_t i = 1;; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(kSuspendNs)
        : "memory");
    if (done) return true;
    // back off: a spinning warp would take issue slots from the working warps of its
    // sub-partition (the copy and MMA warps wait most of the time)
    __nanosleep(sleep_ns);
    if (sleep_ns < 256u) sleep_ns <<= 1;
    if ((i & 15u) == 0 && global_ns() - t0 > kWaitNs) return false;
  }
}
// every lane waits (each wait is bounded, so every lane gets here) and the warp agrees
// on the outcome, so that the warp-collective instructions after it stay uniform
__device__ __forceinline__ bool warp_wait(uint64_t* b, uint32_t parity) {
  return __all_sync(0xffffffffu, wait_phase(b, parity) ? 1 : 0) != 0;
}
__device__ __forceinline__ bool warp_aborted(volatile int* f, int lane) {
  const int v = lane == 0 ? *f : 0;
  return __shfl_sync(0xffffffffu, v, 0) != 0;
}

// The item sequence of one CTA, walked with counters: item k is (tile, Ja) with
// Ja = b + (k mod nJ) G and tile = (b mod T + k div nJ) mod T.
struct Cursor {
  int64_t k = 0, end = 0, j = 0, nJ = 0, b = 0, G = 1, T = 1;
  int64_t tile = 0, Ja = 0;
  int64_t e0 = 0;  // first single of Ja
  int ns = 0;      // singles of Ja
  __device__ void init(int64_t b_, int64_t G_, int64_t Na, int64_t T_) {
    b = b_;
    G = G_;
    T = T_;
    nJ = b < Na ? (Na - b + G - 1) / G : 0;
    end = T * nJ;
    k = 0;
    j = 0;
    tile = b % T;
    Ja = b;
  }
  __device__ void advance() {
    ++k;
    Ja += G;
    if (++j == nJ) {
      j = 0;
      Ja = b;
      if (++tile == T) tile = 0;
    }
  }
  // move to the next item (this one included) whose alpha string has singles
  __device__ bool next(const Args& A) {
    while (k < end) {
      e0 = __ldg(A.a_srow + Ja);
      ns = (int)(__ldg(A.a_srow + Ja + 1) - e0);
      if (ns > 0) return true;
      advance();
    }
    return false;
  }
};

__device__ __forceinline__ int mma_n(int ns) { return ns <= 16 ? 16 : (ns + 15) & ~15; }

__global__ void __launch_bounds__(kThreads, 1) k_sigma_ab_tc2(Args A) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int KB = A.KB, Kp = A.Kp, n = A.n;
  const uint32_t d_bytes = (uint32_t)kTileM * KB * 16;
  const uint32_t bs_bytes = (uint32_t)kMaxSingles * KB * 16;
  unsigned char* sB = smem;                // the folded table
  unsigned char* sBs = smem + A.off_Bs;    // [2] the item's B operand
  unsigned char* sD = smem + A.off_D;      // [2] D
  unsigned char* sC = smem + A.off_C;      // [2] C(Ja, :)
  uint16_t* sF = reinterpret_cast<uint16_t*>(smem + A.off_F);  // [n*n] folded pair
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + A.off_bar);
  uint64_t* crow_full = bar;       // [2] copy of C(Ja, :) landed
  uint64_t* crow_empty = bar + 2;  // [2] gather done reading it (one arrival per warp)
  uint64_t* d_full = bar + 4;      // [2] D and B stages written (one arrival per warp)
  uint64_t* mma_done = bar + 6;    // [2] MMA chain of the stage finished (commit)
  uint64_t* acc_empty = bar + 8;   // [2] epilogue done with the accumulator (per warp)
  uint64_t* cleared = bar + 10;    // [2] D stage cleared for a new tile (per gather warp)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 12);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bar + 12) + 1;

  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(crow_full + s, 1);
      mbar_init(crow_empty + s, kGatherWarps);
      mbar_init(d_full + s, kGatherWarps);
      mbar_init(mma_done + s, 1);
      mbar_init(acc_empty + s, kEpiWarps);
      mbar_init(cleared + s, kGatherWarps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  for (int i = tid; i < Kp * KB; i += kThreads)  // the stationary table
    reinterpret_cast<uint4*>(sB)[i] = __ldg(A.Bimg + i);
  for (int i = tid; i < (int)(2 * d_bytes / 16); i += kThreads)  // D stages start at zero
    reinterpret_cast<uint4*>(sD)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < n * n; i += kThreads) {
    const int p = i / n, q = i - p * n;
    sF[i] = (uint16_t)(p >= q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p);
  }
  fence_proxy_async();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  auto give_up = [&]() {
    ok = false;
    *abort_flag = 1;
    atomicExch(&g_tc_error, 1);
  };
  Cursor cur;
  cur.init(blockIdx.x, gridDim.x, A.Na, A.T);

  if (warp == 0) {
    // --------------------------------------------- C rows into shared stages
    int q = 0;
    for (; ok && !warp_aborted(abort_flag, lane) && cur.next(A); cur.advance(), ++q) {
      const int s = q & 1;
      float* dst = reinterpret_cast<float*>(sC + (size_t)s * A.crow_stride);
      if (q >= 2 && !warp_wait(crow_empty + s, ((q - 2) >> 1) & 1)) {
        if (lane == 0) give_up();
        break;
      }
      const float* src = A.C + cur.Ja * A.Nb;
      if (A.bulk_row) {
        if (lane == 0) {
          mbar_expect_tx(crow_full + s, (uint32_t)(A.Nb * 4));
          bulk_g2s(dst, src, (uint32_t)(A.Nb * 4), crow_full + s);
        }
      } else {
        for (int64_t j = lane; j < A.Nb; j += 32) dst[j] = __ldg(src + j);
        __syncwarp();
        if (lane == 0) mbar_arrive(crow_full + s);
      }
      __syncwarp();
    }
    // copies still in flight land before the CTA can exit
    if (A.bulk_row && lane == 0) {
      for (int k = (q >= 2 ? q - 2 : 0); k < q; ++k) wait_phase(crow_full + (k & 1), (k >> 1) & 1);
    }
  } else if (warp == 1) {
    // --------------------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t sbo = (uint32_t)KB * 128;
      int q = 0;
      for (; ok && !*abort_flag && cur.next(A); cur.advance(), ++q) {
        const int s = q & 1;
        if (!wait_phase(d_full + s, (q >> 1) & 1) ||
            (q >= 2 && !wait_phase(acc_empty + s, ((q - 2) >> 1) & 1))) {
          give_up();
          break;
        }
        fence_after();
        const uint32_t idesc = make_idesc(kTileM, mma_n(cur.ns));
        const uint32_t a0 = smem_u32(sD + (size_t)s * d_bytes);
        const uint32_t b0 = smem_u32(sBs + (size_t)s * bs_bytes);
        const uint32_t d = tmem + (uint32_t)(s * kMaxSingles);
        for (int kk = 0; kk < KB / 2; ++kk) {
          const uint32_t off = (uint32_t)kk * 256;  // 16 K elements = two core matrices
          mma_bf16(d, make_desc(a0 + off, 128, sbo), make_desc(b0 + off, 128, sbo), idesc,
                   kk > 0 ? 1u : 0u);
        }
        mma_commit(smem_u32(mma_done + s));
      }
      // MMAs in flight finish before tensor memory is freed
      for (int k = (q >= 2 ? q - 2 : 0); k < q; ++k) wait_phase(mma_done + (k & 1), (k >> 1) & 1);
    }
  } else if (warp < 2 + kGatherWarps) {
    // ------------------------------------------------------------------ gather
    const int g = tid - 64, gw = g >> 5, m = g & (kTileM - 1), h = g >> 7;  // row m, slots h, h+2..
    unsigned char* rowD = sD + (m >> 3) * (KB * 128) + (m & 7) * 16;
    int64_t tile = -1, stage_tile[2] = {-1, -1};
    int clears[2] = {0, 0};
    uint32_t slot[kMySlots];
    int mine = 0;  // this thread's slots of the row (slots h, h + 2, ...)
    int q = 0;
    for (; ok && !warp_aborted(abort_flag, lane) && cur.next(A); cur.advance(), ++q) {
      const int s = q & 1;
      const int64_t t = cur.tile;
      const int ns = cur.ns;
      // the item's singles (lane u holds singles u and u + 32), read early
      const int sp0 = lane < ns ? __ldg(&A.a_slink[cur.e0 + lane].y) : 1;
      const int sp1 = lane + 32 < ns ? __ldg(&A.a_slink[cur.e0 + lane + 32].y) : 1;
      if (t != tile) {  // this beta string's slots of the new tile
        tile = t;
        const int64_t Ib = t * kTileM + m;
        const int all = Ib < A.Nb ? __ldg(A.b_cnt + Ib) : 0;
        mine = all > h ? (all - h + kThreadsPerRow - 1) / kThreadsPerRow : 0;
#pragma unroll
        for (int i = 0; i < kMySlots; ++i) {
          if (i >= mine) break;
          const int j = kThreadsPerRow * i + h;
          const int2 r = __ldg(A.b_tcell + ((((int64_t)(j >> 1) * A.Nb + Ib) << 1) + (j & 1)));
          slot[i] = (uint32_t)r.x | (((uint32_t)r.y & 0xFFFu) << kSlotJbBits) |
                    ((uint32_t)r.y & 0x80000000u);
        }
      }
      if (q >= 2 && !warp_wait(mma_done + s, ((q - 2) >> 1) & 1)) {
        if (lane == 0) give_up();
        break;
      }
      if (stage_tile[s] != t) {
        // a new tile in this stage: the gather warps clear the stage together (the two
        // threads of a row write the same 16-byte chunks, so every clear must land
        // before any write)
        for (int i = g; i < (int)(d_bytes / 16); i += kGather)
          reinterpret_cast<uint4*>(sD + (size_t)s * d_bytes)[i] = make_uint4(0, 0, 0, 0);
        __syncwarp();
        if (lane == 0) mbar_arrive(cleared + s);
        if (!warp_wait(cleared + s, clears[s] & 1)) {
          if (lane == 0) give_up();
          break;
        }
        ++clears[s];
        stage_tile[s] = t;
      }
      // B stage s: the (pq|.) rows of Ja's singles with the sign folded in, copied from
      // the stationary table; warp gw takes singles gw, gw + 8, ..., lane = 16-byte chunk
      // (rows ns .. N-1 of the MMA are left as they are: the epilogue never reads them)
      unsigned char* bst = sBs + (size_t)s * bs_bytes;
      for (int a0 = gw; a0 < ns; a0 += 4 * kGatherWarps) {  // four singles' loads in flight
        uint4 v[4];
        int sp[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int a = a0 + u * kGatherWarps;
          sp[u] = __shfl_sync(0xffffffffu, a < 32 ? sp0 : sp1, a & 31);
          v[u] = make_uint4(0, 0, 0, 0);
          if (a < ns && lane < KB) {
            const int r = sF[(sp[u] > 0 ? sp[u] : -sp[u]) - 1];
            v[u] = *reinterpret_cast<const uint4*>(sB + (r >> 3) * (KB * 128) + lane * 128 + (r & 7) * 16);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int a = a0 + u * kGatherWarps;
          if (a < ns && lane < KB) {
            uint4 w = v[u];
            if (sp[u] < 0) w.x ^= 0x80008000u, w.y ^= 0x80008000u, w.z ^= 0x80008000u, w.w ^= 0x80008000u;
            *reinterpret_cast<uint4*>(bst + (a >> 3) * (KB * 128) + lane * 128 + (a & 7) * 16) = w;
          }
        }
      }
      if (!warp_wait(crow_full + s, (q >> 1) & 1)) {
        if (lane == 0) give_up();
        break;
      }
      const float* row = reinterpret_cast<const float*>(sC + (size_t)s * A.crow_stride);
      unsigned char* dst = rowD + (size_t)s * d_bytes;
      constexpr uint32_t kJb = (1u << kSlotJbBits) - 1u;
      {  // every load of the item in flight before the stores: one shared-memory latency
        float v[kMySlots];
#pragma unroll
        for (int i = 0; i < kMySlots; ++i) v[i] = i < mine ? row[slot[i] & kJb] : 0.0f;
#pragma unroll
        for (int i = 0; i < kMySlots; ++i)
          if (i < mine)
            *reinterpret_cast<__nv_bfloat16*>(dst + ((slot[i] >> kSlotJbBits) & 0xFFFu)) =
                __float2bfloat16_rn(__uint_as_float(__float_as_uint(v[i]) ^ (slot[i] & 0x80000000u)));
      }
      // each thread's shared-memory writes are made visible to the tensor cores, the
      // warp synchronises, and one lane arrives for the warp
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(crow_empty + s);
        mbar_arrive(d_full + s);
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int quarter = warp & 3;  // the 32 tensor-memory lanes this warp may read
    const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
    const unsigned full = 0xffffffffu;
    int q = 0;
    for (; ok && !warp_aborted(abort_flag, lane) && cur.next(A); cur.advance(), ++q) {
      const int s = q & 1;
      const int ns = cur.ns;
      // target rows of the item's singles (lane u holds singles u and u + 32), read
      // before the wait so that their latency overlaps the MMA
      const int tgt0 = lane < ns ? __ldg(&A.a_slink[cur.e0 + lane].x) : 0;
      const int tgt1 = lane + 32 < ns ? __ldg(&A.a_slink[cur.e0 + lane + 32].x) : 0;
      if (!warp_wait(mma_done + s, (q >> 1) & 1)) {
        if (lane == 0) give_up();
        break;
      }
      fence_after();
      const int64_t ib = cur.tile * kTileM + 32 * quarter + lane;
      const uint32_t acc = tmem + lane_base + (uint32_t)(s * kMaxSingles);
      float* srow = A.sig + ib;
      const bool live = ib < A.Nb;
      // 32 accumulator columns at a time; the accumulator is released after the last read
#pragma unroll
      for (int h0 = 0; h0 < kMaxSingles; h0 += 32) {
        if (h0 >= ns) break;
        float v[32];
        tmem_ld16_nowait(acc + (uint32_t)h0, v);
        if (h0 + 16 < ns) tmem_ld16_nowait(acc + (uint32_t)(h0 + 16), v + 16);
        tmem_wait_ld();
        if (h0 + 32 >= ns) {
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(acc_empty + s);  // the next MMA may start
        }
        const int tg = h0 < 32 ? tgt0 : tgt1;
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int J = __shfl_sync(full, tg, u);
          if (h0 + u < ns && live) atomicAdd(srow + (int64_t)J * A.Nb, v[u]);
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

// Shared-memory image of the folded table: element (row kf_pq, column kf_rs) at the
// K-major core-matrix offset (row / 8) * KB * 128 + (col / 8) * 128 + (row % 8) * 16
// + (col % 8) * 2; rows and columns at or above K are zero.
__global__ void k_bfold(const float* __restrict__ eri32, int n, int K, int KB,
                        __nv_bfloat16* __restrict__ img) {
  const int Kp = KB * 8, n2 = n * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)Kp * Kp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / Kp), k = (int)(i % Kp);
    float v = 0.0f;
    if (r < K && k < K) {
      int p = 0, x = 0;
      while ((p + 1) * (p + 2) / 2 <= r) ++p;
      while ((x + 1) * (x + 2) / 2 <= k) ++x;
      const int q = r - p * (p + 1) / 2, y = k - x * (x + 1) / 2;
      v = eri32[(int64_t)(p * n + q) * n2 + x * n + y];
    }
    const int64_t off = ((int64_t)(r >> 3) * (KB * 128) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2) / 2;
    img[off] = __float2bfloat16_rn(v);
  }
}

static size_t align128(size_t x) { return (x + 127) & ~(size_t)127; }

// kTcNoFit when the problem is outside this kernel's range (the caller falls back)
static int launch(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                  const hinqs_links_s* lb, const float* c, float* sig, cudaStream_t s) {
  if (!H->tc_bfold || B->Nb >= (int64_t(1) << kSlotJbBits) || B->Na == 0 || B->Nb == 0 ||
      la->max_srow > kMaxSingles || lb->ell_width > kMaxSlots)
    return kTcNoFit;
  Args a;
  a.Na = B->Na;
  a.Nb = B->Nb;
  a.T = ceil_div(B->Nb, kTileM);
  a.n = H->n;
  a.KB = H->tc_KB;
  a.Kp = H->tc_KB * 8;
  a.a_srow = la->srow_ptr;
  a.a_slink = la->slink;
  a.b_tcell = lb->tcell;
  a.b_cnt = lb->scount;
  a.Bimg = reinterpret_cast<const uint4*>(H->tc_bfold);
  a.C = c;
  a.sig = sig;
  a.bulk_row = (B->Nb % 4 == 0) && ((reinterpret_cast<uintptr_t>(c) & 15u) == 0);
  const size_t b_bytes = (size_t)a.Kp * a.KB * 16;
  const size_t bs_bytes = (size_t)kMaxSingles * a.KB * 16;
  const size_t d_bytes = (size_t)kTileM * a.KB * 16;
  a.crow_stride = (uint32_t)align128((size_t)B->Nb * 4);
  a.off_Bs = (uint32_t)align128(b_bytes);
  a.off_D = a.off_Bs + (uint32_t)(2 * bs_bytes);
  a.off_C = a.off_D + (uint32_t)(2 * d_bytes);
  a.off_F = a.off_C + 2 * a.crow_stride;
  a.off_bar = (uint32_t)align128(a.off_F + (size_t)H->n * H->n * 2);
  const size_t bytes = a.off_bar + 12 * 8 + 8;
  if (bytes > (size_t)smem_optin_limit()) return kTcNoFit;
  auto kern = k_sigma_ab_tc2;
  HQ_TRY(allow_max_smem(kern));
  // one CTA per SM (the persistent grid covers the SMs once): the request is padded
  // above half of an SM's shared memory
  const size_t req = std::max(bytes, (size_t)120 * 1024);
  int dev = 0, sms = kNumSMs;
  HQ_CUDA(cudaGetDevice(&dev));
  HQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = (int)std::min<int64_t>(B->Na, sms);
  kern<<<grid, kThreads, req, s>>>(a);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

}  // namespace tc2

int tc_tables_build(hinqs_ham_s* H, cudaStream_t s) {
  const int n = H->n;
  if (n > kTcMaxOrb) return HINQS_OK;  // the tensor-core path is not offered
  const int K = n * (n + 1) / 2;
  H->tc_KB = (int)ceil_div(K, 16) * 2;
  const int64_t cnt = (int64_t)n * n * H->tc_KB * 8;
  HQ_TRY(dalloc(&H->tc_bhi, cnt, s));
  HQ_TRY(dalloc(&H->tc_blo, cnt, s));
  tc::k_btable<<<(unsigned)std::min<int64_t>(ceil_div(cnt, 256), 1024), 256, 0, s>>>(
      H->eri32, n, K, H->tc_KB, reinterpret_cast<__nv_bfloat16*>(H->tc_bhi),
      reinterpret_cast<__nv_bfloat16*>(H->tc_blo));
  HQ_LAUNCH_CHECK();
  const int Kp = H->tc_KB * 8;
  if (Kp <= tc2::kMaxKp) {
    HQ_TRY(dalloc(&H->tc_bfold, (int64_t)Kp * Kp, s));
    tc2::k_bfold<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)Kp * Kp, 256), 1024), 256, 0, s>>>(
        H->eri32, n, K, H->tc_KB, reinterpret_cast<__nv_bfloat16*>(H->tc_bfold));
    HQ_LAUNCH_CHECK();
  }
  return HINQS_OK;
}

int sigma_ab_tc_batch(const SigmaReq* reqs, const int* idx, int n, int split, cudaStream_t s) {
  if (n <= 0) return HINQS_OK;
  std::vector<tc::Args> args;
  bool wide = false;
  for (int i = 0; i < n; ++i) {
    const SigmaReq& r = reqs[idx[i]];
    if (!r.H->tc_bhi || r.H->tc_KB != reqs[idx[0]].H->tc_KB) return kTcNoFit;
    tc::Args a;
    a.Na = r.B->Na;
    a.Nb = r.B->Nb;
    a.n = r.H->n;
    a.KB = r.H->tc_KB;
    a.a_srow = r.la->srow_ptr;
    a.a_slink = r.la->slink;
    a.b_ell = r.lb->tcell;
    a.b_q = reinterpret_cast<const uint4*>(r.lb->tcq);
    a.wq = (r.lb->ell_width + 3) >> 2;
    a.b_cnt = r.lb->scount;
    a.Bhi = reinterpret_cast<const uint4*>(r.H->tc_bhi);
    a.Blo = reinterpret_cast<const uint4*>(r.H->tc_blo);
    a.C = static_cast<const float*>(r.x);
    a.sig = static_cast<float*>(r.y);
    a.crow_smem = 0;
    wide = wide || r.la->max_srow > 64;
    args.push_back(a);
  }
  if (split == 3)
    return wide ? tc::launch_batch<128, 3>(args, s) : tc::launch_batch<64, 3>(args, s);
  return wide ? tc::launch_batch<128, 1>(args, s) : tc::launch_batch<64, 1>(args, s);
}

int sigma_ab_tc_launch(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                       const hinqs_links_s* lb, const float* c, float* sig, int split,
                       cudaStream_t s) {
  if (!H->tc_bhi) return kTcNoFit;  // n_orb above kTcMaxOrb
  if (split == 1 && la->tune_stages == 3) {  // the tile-stationary form, when chosen
    const int r2 = tc2::launch(H, B, la, lb, c, sig, s);
    if (r2 != kTcNoFit) return r2;
  }
  tc::Args a;
  a.Na = B->Na;
  a.Nb = B->Nb;
  a.n = H->n;
  a.KB = H->tc_KB;
  a.a_srow = la->srow_ptr;
  a.a_slink = la->slink;
  a.b_ell = lb->tcell;
  a.b_q = reinterpret_cast<const uint4*>(lb->tcq);
  a.wq = (lb->ell_width + 3) >> 2;
  a.b_cnt = lb->scount;
  a.Bhi = reinterpret_cast<const uint4*>(H->tc_bhi);
  a.Blo = reinterpret_cast<const uint4*>(H->tc_blo);
  a.C = c;
  a.sig = sig;
  a.crow_smem = 0;
  // alpha strings with more than 64 singles take 128-column chunks when the tiles fit,
  // else 64-column chunks in several passes; at most 32 singles a string: 32-column
  // chunks (half the MMA and operand work of a 64-column chunk, more CTAs per SM);
  // kTcNoFit when nothing fits
  const bool wide = la->max_srow > 64, narrow = la->max_srow <= 32;
  if (split == 3) {
    if (wide && tc::fits<128, 3>(a)) return tc::launch_fit<128, 3>(a, la->tune_stages, s);
    if (narrow && tc::fits<32, 3>(a)) return tc::launch_fit<32, 3>(a, la->tune_stages, s);
    return tc::fits<64, 3>(a) ? tc::launch_fit<64, 3>(a, la->tune_stages, s) : kTcNoFit;
  }
  if (wide && tc::fits<128, 1>(a)) return tc::launch_fit<128, 1>(a, la->tune_stages, s);
  if (narrow && tc::fits<32, 1>(a)) return tc::launch_fit<32, 1>(a, la->tune_stages, s);
  return tc::fits<64, 1>(a) ? tc::launch_fit<64, 1>(a, la->tune_stages, s) : kTcNoFit;
}

namespace tc {

// Diagnostic for the timeout path: one thread waits, with the sigma kernel's bounded
// wait and `limit` polls, on an mbarrier whose single expected arrival never comes,
// and raises the same error flag when the wait gives up.  Nothing else touches the
// barrier, so the wait always ends by its limit.
__global__ void k_wait_selftest(long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(smem_u32(&bar), 0u, limit)) atomicExch(&g_tc_error, 1);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
  }
}

}  // namespace tc

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

extern "C" int hinqs_selftest_bounded_wait(long long polls, void* stream) {
  if (polls < 1 || polls > hinqs::tc::kWaitLimit)
    return hinqs::fail(HINQS_ERR_ARG, "hinqs_selftest_bounded_wait: polls outside 1..2^26");
  cudaStream_t s = (cudaStream_t)stream;
  hinqs::tc::k_wait_selftest<<<1, 32, 0, s>>>(polls);
  HQ_LAUNCH_CHECK();
  return hinqs::tc_error_check(s);
}
