// K9: spin-summed 1- and 2-RDMs of a state on the product subspace (FP64 results;
// the string-pair weights and the opposite-spin sums in double-float arithmetic, about
// 1e-13 relative), the Hellmann-Feynman gradients of the energy;
// K10: spin marginals (Step 4).
//
//   gamma_pq   = sum_s <a+_ps a_qs>
//   Gamma_pqrs = sum_{s,t} <a+_ps a+_rt a_st a_qs>
//              = G^aa + G^bb + G^ab_pqrs + G^ab_rspq,  G^ab_pqrs = <E^a_pq E^b_rs>
//
// Same-spin parts come from the string-pair weights
//   M_a(I,J) = sum_b c(I,b) c(J,b),   M_b(I,J) = sum_a c(a,I) c(a,J)
// on the linked pairs (and I = J), expanded with the index patterns of the
// one- and two-body transition elements between strings.  The opposite-spin
// part groups the beta transitions (bra I_b, ket J_b, pair rs, sign) by rs and,
// per ket alpha string J_a and alpha transition (I_a, pq, sign), sums
//   X[pq][rs] = sum_{(I_b,J_b,s_b) with pair rs} s_b c(I_a,I_b) c(J_a,J_b).
#include <algorithm>

#include "hinqs_internal.cuh"

namespace hinqs {

// X2[i] = (hi, lo) double-float pair of X[i]
__global__ void k_df_split(const double* __restrict__ X, int64_t m, float2* __restrict__ X2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    X2[i] = df_split(X[i]);
}

// (sh, sl) += a * b in double-float with the two cross terms rounded separately and
// then added, so that swapping a and b gives the same bits (M(I, J) = M(J, I))
__device__ __forceinline__ void df_fma_sym(float2 a, float2 b, float& sh, float& sl) {
  const float p = a.x * b.x;
  const float e = fmaf(a.x, b.x, -p) + (a.x * b.y + a.y * b.x);
  df_add(p, e, sh, sl);
}

// M[k] = dot(row_I, row_J) for every link k (I -> J = col[k]) of the rows of X
// (n_rows x len, double-float pairs), plus Mdiag[I] = |row_I|^2; one warp per row, the
// sums as double-float pairs (FP64 runs at 1/64 of the FP32 rate on this part, and
// these dot products are the bulk of the same-spin RDM work).
__global__ void k_link_dots_df(const float2* __restrict__ X, int64_t len,
                               const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               int64_t nrows, double* __restrict__ M, double* __restrict__ Mdiag) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  auto reduce = [&](float h, float l) {
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_down_sync(full, h, o), ol = __shfl_down_sync(full, l, o);
      df_add(oh, ol, h, l);
    }
    return (double)h + (double)l;
  };
  for (int64_t I = warp; I < nrows; I += nw) {
    const float2* xi = X + I * len;
    float dh = 0.f, dl = 0.f;
    for (int64_t j = lane; j < len; j += 32) df_fma_sym(xi[j], xi[j], dh, dl);
    const double d = reduce(dh, dl);
    if (lane == 0) Mdiag[I] = d;
    for (int64_t k = rp[I]; k < rp[I + 1]; ++k) {
      const float2* xj = X + (int64_t)col[k] * len;
      float vh = 0.f, vl = 0.f;
      for (int64_t j = lane; j < len; j += 32) df_fma_sym(xi[j], xj[j], vh, vl);
      const double v = reduce(vh, vl);
      if (lane == 0) M[k] = v;
    }
  }
}

// Tiled transpose: out[j][i] = in[i][j] for in of rows x cols.
__global__ void k_transpose(const double* __restrict__ in, double* __restrict__ out, int64_t rows,
                            int64_t cols) {
  __shared__ double tile[32][33];
  int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int64_t i = by + k, j = bx + threadIdx.x;
    if (i < rows && j < cols) tile[k][threadIdx.x] = in[i * cols + j];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int64_t j = bx + k, i = by + threadIdx.x;
    if (i < rows && j < cols) out[j * rows + i] = tile[threadIdx.x][k];
  }
}

// Same-spin contributions of one species into g1 (n^2) and g2 (n^4).
// Row J is the ket; each link record gives the bra I = col with
// <I| a+_p a_q |J> = sign (single) or <I| a+_p a+_r a_s a_q |J> = sign (double).
__global__ void k_same_spin_expand(const uint64_t* __restrict__ S, int64_t N, int n,
                                   const int64_t* __restrict__ rp, const uint32_t* __restrict__ exc,
                                   const int8_t* __restrict__ sign, const int8_t* __restrict__ degree,
                                   const double* __restrict__ M, const double* __restrict__ Mdiag,
                                   double* __restrict__ g1, double* __restrict__ g2) {
  const int64_t n2 = (int64_t)n * n, n3 = n2 * n;
  auto G2 = [&](int p, int q, int r, int s, double v) {
    if (g2) atomicAdd(g2 + p * n3 + q * n2 + (int64_t)r * n + s, v);
  };
  for (int64_t J = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; J < N;
       J += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t x = S[J];
    const double md = Mdiag[J];
    // diagonal: gamma_qq += M; Gamma_qqss += M, Gamma_sqqs -= M for q != s in J
    uint64_t oq = x;
    while (oq) {
      int q = __ffsll((long long)oq) - 1;
      oq &= oq - 1;
      atomicAdd(g1 + q * n + q, md);
      uint64_t os = x;
      while (os) {
        int s = __ffsll((long long)os) - 1;
        os &= os - 1;
        if (s == q) continue;
        G2(q, q, s, s, md);
        G2(s, q, q, s, -md);
      }
    }
    for (int64_t k = rp[J]; k < rp[J + 1]; ++k) {
      const uint32_t e = exc[k];
      const int p = e & 255, q = (e >> 8) & 255, r = (e >> 16) & 255, s = e >> 24;
      const double v = sign[k] * M[k];
      if (degree[k] == 1) {
        // bra = sign a+_p a_q |J>, particle e = p, hole h = q, spectators k in J \ {q}
        atomicAdd(g1 + p * n + q, v);
        uint64_t ok = x & ~(1ull << q);
        while (ok) {
          int kk = __ffsll((long long)ok) - 1;
          ok &= ok - 1;
          G2(p, q, kk, kk, v);
          G2(kk, q, p, kk, -v);
          G2(p, kk, kk, q, -v);
          G2(kk, kk, p, q, v);
        }
      } else {
        G2(p, q, r, s, v);
        G2(r, q, p, s, -v);
        G2(p, s, r, q, -v);
        G2(r, s, p, q, v);
      }
    }
  }
}

// Beta transitions grouped by pair rs: count, then place.
// Transition (bra I_b, ket J_b, rs, s_b): from ket row J_b's single links
// (bra = col, rs = p*n+q, sign) and the diagonal (I_b = J_b, rs = jj, +1).
__global__ void k_trans_count(const uint64_t* __restrict__ S, int64_t N, int n,
                              const int64_t* __restrict__ srp, const int2* __restrict__ sl,
                              int64_t* __restrict__ cnt) {
  for (int64_t J = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; J < N;
       J += (int64_t)gridDim.x * blockDim.x) {
    uint64_t o = S[J];
    while (o) {
      int j = __ffsll((long long)o) - 1;
      o &= o - 1;
      atomicAdd((unsigned long long*)(cnt + j * n + j), 1ull);
    }
    for (int64_t k = srp[J]; k < srp[J + 1]; ++k) {
      int sp = sl[k].y;
      int rs = (sp > 0 ? sp : -sp) - 1;
      atomicAdd((unsigned long long*)(cnt + rs), 1ull);
    }
  }
}

__global__ void k_trans_place(const uint64_t* __restrict__ S, int64_t N, int n,
                              const int64_t* __restrict__ srp, const int2* __restrict__ sl,
                              int64_t* __restrict__ cursor, int4* __restrict__ out) {
  for (int64_t J = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; J < N;
       J += (int64_t)gridDim.x * blockDim.x) {
    uint64_t o = S[J];
    while (o) {
      int j = __ffsll((long long)o) - 1;
      o &= o - 1;
      int64_t pos = (int64_t)atomicAdd((unsigned long long*)(cursor + j * n + j), 1ull);
      out[pos] = make_int4((int)J, (int)J, 1, 0);
    }
    for (int64_t k = srp[J]; k < srp[J + 1]; ++k) {
      int2 l = sl[k];
      int rs = (l.y > 0 ? l.y : -l.y) - 1;
      int64_t pos = (int64_t)atomicAdd((unsigned long long*)(cursor + rs), 1ull);
      out[pos] = make_int4(l.x, (int)J, l.y > 0 ? 1 : -1, 0);
    }
  }
}

// Opposite-spin 2-RDM for rows too long to stage, one block per ket alpha string J_a;
// CH alpha transitions at a time; thread per (transition, rs) bin, the rows read from
// the double-float copy of C and the sum kept as a double-float pair.
template <int CH>
__global__ void __launch_bounds__(256) k_rdm_ab_df(const float2* __restrict__ C2, int64_t Nb, int n,
                                                const uint64_t* __restrict__ Sa,
                                                const int64_t* __restrict__ a_srp,
                                                const int2* __restrict__ a_sl,
                                                const int64_t* __restrict__ off,
                                                const int4* __restrict__ trans,
                                                double* __restrict__ gab) {
  const int n2 = n * n;
  const int64_t Ja = blockIdx.x;
  __shared__ int tI[CH], tpq[CH], ts[CH];
  // alpha transitions of ket J_a: diagonal (I = J, pq = ii) then single links
  const uint64_t x = Sa[Ja];
  const int nd = __popcll(x);
  const int64_t nl = a_srp[Ja + 1] - a_srp[Ja];
  const int64_t total = nd + nl;
  const float2* cj = C2 + Ja * Nb;
  for (int64_t t0 = 0; t0 < total; t0 += CH) {
    const int cnt = (int)min64(CH, total - t0);
    __syncthreads();
    if (threadIdx.x < cnt) {
      int64_t t = t0 + threadIdx.x;
      if (t < nd) {
        // t-th occupied orbital of J_a
        uint64_t o = x;
        for (int k = 0; k < t; ++k) o &= o - 1;
        int i = __ffsll((long long)o) - 1;
        tI[threadIdx.x] = (int)Ja;
        tpq[threadIdx.x] = i * n + i;
        ts[threadIdx.x] = 1;
      } else {
        int2 l = a_sl[a_srp[Ja] + (t - nd)];
        tI[threadIdx.x] = l.x;
        tpq[threadIdx.x] = (l.y > 0 ? l.y : -l.y) - 1;
        ts[threadIdx.x] = l.y > 0 ? 1 : -1;
      }
    }
    __syncthreads();
    for (int bin = threadIdx.x; bin < cnt * n2; bin += blockDim.x) {
      const int a = bin / n2, rs = bin % n2;
      const float2* ci = C2 + (int64_t)tI[a] * Nb;
      float ah = 0.f, al = 0.f;
      for (int64_t k = off[rs]; k < off[rs + 1]; ++k) {
        const int4 tr = trans[k];
        const float2 x = ci[tr.x];
        float2 y = cj[tr.y];
        if (tr.z < 0) y.x = -y.x, y.y = -y.y;
        df_fma(x.x, x.y, y.x, y.y, ah, al);
      }
      const double acc = (double)ah + (double)al;
      if (acc != 0.0) atomicAdd(gab + (int64_t)tpq[a] * n2 + rs, ts[a] * acc);
    }
  }
}

// Opposite-spin 2-RDM with the rows staged in shared memory.  Block (J_a, chunk):
// up to U alpha transitions (I_a, pq, s_a) of the ket J_a (diagonal first, then the
// single links); the bra rows C(I_a, :) of the chunk and the ket row C(J_a, :) are
// copied to shared memory.  The beta transitions, grouped by pair rs, are cut into
// segments of at most kRdmSeg entries so that the lanes of a warp carry equal work;
// a thread walks a segment once and updates U accumulators, one double-float
// multiply-add per term (C split once into (hi, lo) FP32 pairs, the same eight bytes an
// element as in FP64):
//   X[u][rs] += C(I_a,u, I_b) * s_b C(J_a, J_b),
// then adds s_a X[u][rs] into gab[pq_u][rs] (FP64).
constexpr int kRdmSeg = 128;

__global__ void k_seg_count(const int64_t* __restrict__ off, int n2, int64_t* __restrict__ cnt) {
  for (int rs = blockIdx.x * blockDim.x + threadIdx.x; rs < n2; rs += gridDim.x * blockDim.x)
    cnt[rs] = (off[rs + 1] - off[rs] + kRdmSeg - 1) / kRdmSeg;
}
__global__ void k_seg_fill(const int64_t* __restrict__ off, int n2,
                           const int64_t* __restrict__ sstart, int4* __restrict__ seg) {
  for (int rs = blockIdx.x * blockDim.x + threadIdx.x; rs < n2; rs += gridDim.x * blockDim.x) {
    int64_t b = off[rs], q = sstart[rs];
    for (; b < off[rs + 1]; b += kRdmSeg, ++q)
      seg[q] = make_int4(rs, (int)(b - off[rs]), (int)min64(kRdmSeg, off[rs + 1] - b), 0);
  }
}

template <int U>
__global__ void __launch_bounds__(256) k_rdm_ab_staged_df(
    const float2* __restrict__ C2, int64_t Nb, int n, const uint64_t* __restrict__ Sa,
    const int64_t* __restrict__ a_srp, const int2* __restrict__ a_sl,
    const int64_t* __restrict__ off, const int4* __restrict__ trans,
    const int4* __restrict__ seg, int64_t nseg, double* __restrict__ gab) {
  extern __shared__ __align__(16) float2 sm2[];  // crow[Nb], rows[U][Nb]
  __shared__ int tI[U], tpq[U], ts[U];
  const int n2 = n * n;
  const int64_t Ja = blockIdx.x;
  const uint64_t x = Sa[Ja];
  const int nd = __popcll(x);
  const int64_t total = nd + (a_srp[Ja + 1] - a_srp[Ja]);
  const int64_t t0 = (int64_t)blockIdx.y * U;
  if (t0 >= total) return;
  const int cnt = (int)min64(U, total - t0);
  if (threadIdx.x < U) {
    const int64_t t = t0 + threadIdx.x;
    int I = (int)Ja, pq = 0, sg = 0;  // unused slots: zero sign, row J_a
    if (threadIdx.x < cnt) {
      if (t < nd) {
        uint64_t o = x;
        for (int k = 0; k < t; ++k) o &= o - 1;
        const int i = __ffsll((long long)o) - 1;
        pq = i * n + i;
        sg = 1;
      } else {
        const int2 l = a_sl[a_srp[Ja] + (t - nd)];
        I = l.x;
        pq = (l.y > 0 ? l.y : -l.y) - 1;
        sg = l.y > 0 ? 1 : -1;
      }
    }
    tI[threadIdx.x] = I;
    tpq[threadIdx.x] = pq;
    ts[threadIdx.x] = sg;
  }
  __syncthreads();
  float2* crow = sm2;
  float2* rows = sm2 + Nb;
  for (int64_t j = threadIdx.x; j < Nb; j += blockDim.x) crow[j] = C2[Ja * Nb + j];
  for (int u = 0; u < U; ++u) {
    const float2* src = C2 + (int64_t)tI[u] * Nb;
    for (int64_t j = threadIdx.x; j < Nb; j += blockDim.x) rows[u * Nb + j] = src[j];
  }
  __syncthreads();
  for (int64_t q = threadIdx.x; q < nseg; q += blockDim.x) {
    const int4 sgm = seg[q];
    const int rs = sgm.x;
    const int4* __restrict__ tr = trans + off[rs] + sgm.y;
    float ah[U], al[U];
#pragma unroll
    for (int u = 0; u < U; ++u) ah[u] = 0.f, al[u] = 0.f;
    for (int k = 0; k < sgm.z; ++k) {
      const int4 t = tr[k];  // {bra I_b, ket J_b, s_b}
      float2 cj = crow[t.y];
      if (t.z < 0) cj.x = -cj.x, cj.y = -cj.y;
      const float2* rb = rows + t.x;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float2 r = rb[u * Nb];
        df_fma(r.x, r.y, cj.x, cj.y, ah[u], al[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const double v = (double)ah[u] + (double)al[u];
      if (u < cnt && v != 0.0) atomicAdd(gab + (int64_t)tpq[u] * n2 + rs, ts[u] * v);
    }
  }
}

__global__ void k_rdm2_combine(const double* __restrict__ same, const double* __restrict__ gab,
                               int n, double* __restrict__ out) {
  const int64_t n2 = (int64_t)n * n, n4 = n2 * n2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t pq = i / n2, rs = i % n2;
    out[i] = same[i] + gab[i] + gab[rs * n2 + pq];
  }
}

__global__ void k_scale(const double* __restrict__ x, double a, double* __restrict__ y, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// ------------------------------------------------------------- marginals --

// row sums of c^2: pa[a] (one block per row)
__global__ void k_row_sq(const double* __restrict__ C, int64_t Na, int64_t Nb, double* pa) {
  __shared__ double red[32];
  for (int64_t a = blockIdx.x; a < Na; a += gridDim.x) {
    double acc = 0.0;
    for (int64_t b = threadIdx.x; b < Nb; b += blockDim.x) {
      double v = C[a * Nb + b];
      acc += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
      pa[a] = v;
    }
    __syncthreads();
  }
}

// column sums of c^2 over a chunk of rows: part[chunk][b]
__global__ void k_col_sq(const double* __restrict__ C, int64_t Na, int64_t Nb, int64_t rows_per,
                         double* part) {
  int64_t chunk = blockIdx.y;
  int64_t a0 = chunk * rows_per, a1 = min64(Na, a0 + rows_per);
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < Nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t a = a0; a < a1; ++a) {
      double v = C[a * Nb + b];
      acc += v * v;
    }
    part[chunk * Nb + b] = acc;
  }
}

__global__ void k_sum_chunks(const double* __restrict__ part, int64_t chunks, int64_t Nb, double* pb) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < Nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t k = 0; k < chunks; ++k) acc += part[k * Nb + b];
    pb[b] = acc;
  }
}

// tot[0] = sum pa (= |c|^2); then normalise pa, pb, and tot[1] = sum pa' * sum pb'
__global__ void k_marg_norm(double* pa, int64_t Na, double* pb, int64_t Nb, double* tot) {
  __shared__ double red[32];
  __shared__ double z;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < Na; i += blockDim.x) acc += pa[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    z = v;
    tot[0] = v;
  }
  __syncthreads();
  const double inv = 1.0 / z;
  double sa = 0.0, sb = 0.0;
  for (int64_t i = threadIdx.x; i < Na; i += blockDim.x) {
    pa[i] *= inv;
    sa += pa[i];
  }
  for (int64_t i = threadIdx.x; i < Nb; i += blockDim.x) {
    pb[i] *= inv;
    sb += pb[i];
  }
  __syncthreads();
  for (int o = 16; o > 0; o >>= 1) sa += __shfl_down_sync(0xffffffffu, sa, o);
  for (int o = 16; o > 0; o >>= 1) sb += __shfl_down_sync(0xffffffffu, sb, o);
  __shared__ double ra[32], rb[32];
  if ((threadIdx.x & 31) == 0) {
    ra[threadIdx.x >> 5] = sa;
    rb[threadIdx.x >> 5] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double A = 0.0, Bv = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      A += ra[w];
      Bv += rb[w];
    }
    tot[1] = A * Bv;
  }
}

__global__ void k_teacher(const double* __restrict__ pa, const double* __restrict__ pb, int64_t Na,
                          int64_t Nb, const double* __restrict__ tot, double* __restrict__ w) {
  const double inv = 1.0 / tot[1];
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < Na * Nb;
       I += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = I / Nb, b = I - a * Nb;
    w[I] = pa[a] * pb[b] * inv;
  }
}

}  // namespace hinqs

using namespace hinqs;

extern "C" int hinqs_rdm(const hinqs_subspace* B, const hinqs_links* la, const hinqs_links* lb,
                         const double* c, double* rdm1, double* rdm2, void* stream) {
  if (!B || !la || !lb) return fail(HINQS_ERR_ARG, "hinqs_rdm: NULL handle");
  if (!c || !rdm1) return fail(HINQS_ERR_ARG, "hinqs_rdm: NULL c or rdm1");
  if (la->spin != 0 || lb->spin != 1 || la->N != B->Na || lb->N != B->Nb ||
      la->strings != B->sa || lb->strings != B->sb)
    return fail(HINQS_ERR_ARG, "hinqs_rdm: links do not belong to this subspace");
  cudaStream_t s = (cudaStream_t)stream;
  const int n = B->n;
  const int64_t n2 = (int64_t)n * n, n4 = n2 * n2, Na = B->Na, Nb = B->Nb, N = Na * Nb;
  double *Ma = nullptr, *Mad = nullptr, *Mb = nullptr, *Mbd = nullptr, *CT = nullptr,
         *same = nullptr, *gab = nullptr;
  float2 *C2 = nullptr, *CT2 = nullptr;  // double-float copies of C and C^T
  int64_t *cnt = nullptr, *off = nullptr;
  int4* trans = nullptr;
  auto cleanup = [&]() {
    dfree(Ma, s);
    dfree(Mad, s);
    dfree(Mb, s);
    dfree(Mbd, s);
    dfree(CT, s);
    dfree(C2, s);
    dfree(CT2, s);
    dfree(same, s);
    dfree(gab, s);
    dfree(cnt, s);
    dfree(off, s);
    dfree(trans, s);
  };
  int rc = HINQS_OK;
  const int64_t ntrans = lb->nsingle + Nb * B->n_beta;
  if ((rc = dalloc(&Ma, la->nnz, s)) || (rc = dalloc(&Mad, Na, s)) || (rc = dalloc(&Mb, lb->nnz, s)) ||
      (rc = dalloc(&Mbd, Nb, s)) || (rc = dalloc(&CT, N, s)) || (rc = dalloc(&C2, N, s)) ||
      (rc = dalloc(&CT2, N, s)) || (rc = dalloc(&same, n4, s)) ||
      (rc = dalloc(&gab, n4, s)) || (rc = dalloc(&cnt, n2 + 1, s)) || (rc = dalloc(&off, n2 + 1, s)) ||
      (rc = dalloc(&trans, ntrans, s))) {
    cleanup();
    return rc;
  }
  auto run = [&]() -> int {
    const int g = 16 * kNumSMs;
    // string-pair weights (double-float rows of C and C^T)
    dim3 tb(32, 8), tg((unsigned)ceil_div(Nb, 32), (unsigned)ceil_div(Na, 32));
    k_transpose<<<tg, tb, 0, s>>>(c, CT, Na, Nb);
    const unsigned gs = (unsigned)std::min<int64_t>(ceil_div(N, 256), 8 * kNumSMs);
    k_df_split<<<gs, 256, 0, s>>>(c, N, C2);
    k_df_split<<<gs, 256, 0, s>>>(CT, N, CT2);
    k_link_dots_df<<<g, 256, 0, s>>>(C2, Nb, la->row_ptr, la->col, Na, Ma, Mad);
    k_link_dots_df<<<g, 256, 0, s>>>(CT2, Na, lb->row_ptr, lb->col, Nb, Mb, Mbd);
    HQ_CUDA(cudaMemsetAsync(rdm1, 0, n2 * sizeof(double), s));
    HQ_CUDA(cudaMemsetAsync(same, 0, n4 * sizeof(double), s));
    HQ_CUDA(cudaMemsetAsync(gab, 0, n4 * sizeof(double), s));
    double* g2 = rdm2 ? same : nullptr;
    k_same_spin_expand<<<(unsigned)std::min<int64_t>(ceil_div(Na, 128), g), 128, 0, s>>>(
        la->strings, Na, n, la->row_ptr, la->exc, la->sign, la->degree, Ma, Mad, rdm1, g2);
    k_same_spin_expand<<<(unsigned)std::min<int64_t>(ceil_div(Nb, 128), g), 128, 0, s>>>(
        lb->strings, Nb, n, lb->row_ptr, lb->exc, lb->sign, lb->degree, Mb, Mbd, rdm1, g2);
    HQ_LAUNCH_CHECK();
    if (!rdm2) return HINQS_OK;
    // beta transitions grouped by rs
    HQ_CUDA(cudaMemsetAsync(cnt, 0, (n2 + 1) * sizeof(int64_t), s));
    k_trans_count<<<(unsigned)std::min<int64_t>(ceil_div(Nb, 128), g), 128, 0, s>>>(
        lb->strings, Nb, n, lb->srow_ptr, lb->slink, cnt);
    int64_t tot = 0;
    HQ_TRY(exclusive_scan_i64(cnt, off, n2 + 1, &tot, s));
    if (tot != ntrans) return fail(HINQS_ERR_CUDA, "hinqs_rdm: transition count mismatch");
    HQ_CUDA(cudaMemcpyAsync(cnt, off, (n2 + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    k_trans_place<<<(unsigned)std::min<int64_t>(ceil_div(Nb, 128), g), 128, 0, s>>>(
        lb->strings, Nb, n, lb->srow_ptr, lb->slink, cnt, trans);
    // staged form when at least four bra rows and the ket row fit in shared memory
    const size_t lim = (size_t)smem_optin_limit();
    const int max_t = B->n_alpha + la->max_srow;  // alpha transitions of one ket
    int U = 0;
    for (int u : {16, 8, 4})
      if ((size_t)(u + 1) * Nb * sizeof(double) + 1024 <= lim && U == 0) U = u;
    if (U) {
      int64_t nseg = 0;
      HQ_CUDA(cudaMemsetAsync(cnt, 0, (n2 + 1) * sizeof(int64_t), s));
      k_seg_count<<<(unsigned)ceil_div(n2, 256), 256, 0, s>>>(off, (int)n2, cnt);
      int64_t* sstart = nullptr;
      int4* seg = nullptr;
      auto staged = [&]() -> int {
        HQ_TRY(dalloc(&sstart, n2 + 1, s));
        HQ_TRY(exclusive_scan_i64(cnt, sstart, n2 + 1, &nseg, s));
        HQ_TRY(dalloc(&seg, std::max<int64_t>(nseg, 1), s));
        k_seg_fill<<<(unsigned)ceil_div(n2, 256), 256, 0, s>>>(off, (int)n2, sstart, seg);
        const dim3 grid((unsigned)Na, (unsigned)ceil_div(max_t, U));
        const size_t smem = (size_t)(U + 1) * Nb * sizeof(double);
        auto go = [&](auto kern) -> int {
          HQ_TRY(allow_max_smem(kern));
          kern<<<grid, 256, smem, s>>>(C2, Nb, n, la->strings, la->srow_ptr, la->slink, off,
                                       trans, seg, nseg, gab);
          return HINQS_OK;
        };
        return U == 16 ? go(k_rdm_ab_staged_df<16>) : U == 8 ? go(k_rdm_ab_staged_df<8>)
                                                             : go(k_rdm_ab_staged_df<4>);
      };
      const int r3 = staged();
      dfree(sstart, s);
      dfree(seg, s);
      HQ_TRY(r3);
    } else {
      k_rdm_ab_df<16><<<(unsigned)Na, 256, 0, s>>>(C2, Nb, n, la->strings, la->srow_ptr,
                                                    la->slink, off, trans, gab);
    }
    k_rdm2_combine<<<(unsigned)std::min<int64_t>(ceil_div(n4, 256), g), 256, 0, s>>>(same, gab, n,
                                                                                   rdm2);
    HQ_LAUNCH_CHECK();
    return HINQS_OK;
  };
  rc = run();
  cleanup();
  return rc;
}

extern "C" int hinqs_energy_backward(int n_orb, double grad_E, const double* rdm1,
                                     const double* rdm2, double* grad_h, double* grad_eri,
                                     void* stream) {
  if (n_orb < 1 || n_orb > 64 || !rdm1 || !grad_h || (grad_eri && !rdm2))
    return fail(HINQS_ERR_ARG, "hinqs_energy_backward: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n2 = (int64_t)n_orb * n_orb, n4 = n2 * n2;
  k_scale<<<(unsigned)std::min<int64_t>(ceil_div(n2, 256), 64), 256, 0, s>>>(rdm1, grad_E, grad_h, n2);
  if (grad_eri)
    k_scale<<<(unsigned)std::min<int64_t>(ceil_div(n4, 256), 4096), 256, 0, s>>>(rdm2, 0.5 * grad_E,
                                                                                grad_eri, n4);
  HQ_LAUNCH_CHECK();
  return HINQS_OK;
}

extern "C" int hinqs_spin_marginals(const hinqs_subspace* B, const double* c, double* pa,
                                    double* pb, double* w, void* stream) {
  if (!B || !c || !pa || !pb) return fail(HINQS_ERR_ARG, "hinqs_spin_marginals: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t Na = B->Na, Nb = B->Nb;
  const int64_t rows_per = 64;
  const int64_t chunks = ceil_div(Na, rows_per);
  double *part = nullptr, *tot = nullptr;
  int rc = HINQS_OK;
  if ((rc = dalloc(&part, chunks * Nb, s)) || (rc = dalloc(&tot, 2, s))) {
    dfree(part, s);
    dfree(tot, s);
    return rc;
  }
  k_row_sq<<<(unsigned)std::min<int64_t>(Na, 16 * kNumSMs), 256, 0, s>>>(c, Na, Nb, pa);
  dim3 g((unsigned)std::min<int64_t>(ceil_div(Nb, 256), 64), (unsigned)chunks);
  k_col_sq<<<g, 256, 0, s>>>(c, Na, Nb, rows_per, part);
  k_sum_chunks<<<(unsigned)std::min<int64_t>(ceil_div(Nb, 256), 256), 256, 0, s>>>(part, chunks, Nb, pb);
  k_marg_norm<<<1, 1024, 0, s>>>(pa, Na, pb, Nb, tot);
  if (w)
    k_teacher<<<(unsigned)std::min<int64_t>(ceil_div(Na * Nb, 256), 16 * kNumSMs), 256, 0, s>>>(
        pa, pb, Na, Nb, tot, w);
  cudaError_t e = cudaGetLastError();
  dfree(part, s);
  dfree(tot, s);
  if (e != cudaSuccess) return cuda_fail(e, "hinqs_spin_marginals", __FILE__, __LINE__);
  return HINQS_OK;
}
