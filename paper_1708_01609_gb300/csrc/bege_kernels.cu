// CUDA kernels of libbege (sm_103a).
//
// Matched filtering by FFT (van Putten, arXiv:1708.01609, Eq. 3S): for a
// real segment y (N samples) and a real template w (L <= N samples,
// zero-padded),
//     rho[n] = sum_m w[m] y[(n+m) mod N]               (Eq. A1, circular)
//            = (1/N) sum_j conj(W_j) D_j e^{+2 pi i j n/N}
// with sigma predicted by Parseval (Eq. PT) and tails |rho| > kappa sigma
// (Eq. tail).
//
// Real transforms as half-length complex transforms.  With H = N/2 and
// z[m] = w[2m] + i w[2m+1], Z = DFT_H(z) gives the template spectrum
//     W_j = (Z_j + conj Z_{H-j})/2 - (i/2) wN^j (Z_j - conj Z_{H-j}).
// The output is packed the same way, yo[n] = rho[2n] + i rho[2n+1], whose
// H-point spectrum is
//     Y_j = (P_j + conj P_{H-j})/2 + (i/2) wN^-j (P_j - conj P_{H-j}),
// P_j = conj(W_j) D_j.  Substituting W gives
//     Y_j = conj(Z_j) A_j + Z_{H-j} B_j,
//     A_j = g_j^2 D_j + d_j^2 conj D_{H-j},  B_j = g_j d_j (D_j + conj D_{H-j}),
//     g_j = (1 + i wN^-j)/2,  d_j = (1 - i wN^-j)/2,
// where A, B depend on the segment only and are computed once per segment
// (segment_kernel).  By Parseval on the packed spectrum
//     sigma^2 = (1/N) sum_n rho_n^2 = 2 sum_{j<H} |Y_j|^2 / N^2,
// the same quantity as Eq. PT's sum over the spectrum of rho.
//
// Residue columns (four-step with a pruned first step).  Bin j = S a + b,
// a < F, b < S, H = S F.  Forward:
//     Z_{Sa+b} = FFT_F(u_b)[a],  u_b[m1] = wH^(b m1) sum_{m2<S} z[m1+F m2] wS^(b m2);
// a template of L <= 2F samples has z = 0 beyond F, so only m2 = 0 remains.
// Inverse: with n = n1 + F n2,
//     yo[n1 + F n2] = (1/H) sum_b wS^(-b n2) T_b[n1],
//     T_b[n1] = wH^(-b n1) IFFT_F(Y_{S.+b})[n1].
// Column b pairs with column S-b (bins j and H-j); columns {0, S/2} and
// {i, S-i} form units.  A CTA owns whole units; the C CTAs of a cluster hold
// all S columns and read each other's columns through distributed shared
// memory only in the final S-point combine.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bege_fft.cuh"
#include "bege_internal.h"

namespace cg = cooperative_groups;

namespace bege {

Geometry make_geometry(int64_t n) {
  Geometry g{};
  g.N = (int)n;
  g.H = g.N / 2;
  g.F = g.H < 4096 ? g.H : 4096;
  g.S = g.H / g.F;
  g.R0 = g.F / 256;
  g.C = g.S >= 8 ? g.S / 4 : 1;
  g.NC = g.S == 1 ? 1 : g.S / g.C;
  const int units = g.S == 1 ? 1 : g.S / 2;
  g.UPC = units / g.C;
  return g;
}

// ---------------------------------------------------------------------------
// Shared-memory layout: compile-time offsets for (F, NC) so every access is
// a shared-memory instruction with an immediate offset.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <int F, int NC>
struct Lay {
  static constexpr int CS = col_stride<F>();
  static constexpr size_t cols = 0;
  static constexpr size_t tw3 = cols + align16(size_t(NC) * CS * 8);
  static constexpr size_t tw2 = tw3 + align16(size_t(F) * 8);
  static constexpr size_t twin = tw2 + align16(256 * 8);
  static constexpr size_t rin = twin + align16(size_t(NC) * 256 * 8);
  static constexpr size_t rout = rin + align16(size_t(NC) * 16 * 8);
  static constexpr size_t ws = rout + align16(size_t(NC) * 16 * 8);
  static constexpr size_t colptr = ws + align16(16 * 8);
  static constexpr size_t red = colptr + align16(16 * 8);
  static constexpr size_t sigpart = red + align16(32 * 4);
  static constexpr size_t slotb = sigpart + align16(4);
  static constexpr size_t total = slotb + align16(4 * 4);
};

extern __shared__ __align__(16) unsigned char smem_raw[];

template <int F, int NC>
struct Smem {
  using L = Lay<F, NC>;
  static __device__ __forceinline__ float2* cols() { return reinterpret_cast<float2*>(smem_raw + L::cols); }
  static __device__ __forceinline__ float2* col(int c) { return cols() + c * L::CS; }
  static __device__ __forceinline__ float2* tw3() { return reinterpret_cast<float2*>(smem_raw + L::tw3); }
  static __device__ __forceinline__ float2* tw2() { return reinterpret_cast<float2*>(smem_raw + L::tw2); }
  static __device__ __forceinline__ float2* twin() { return reinterpret_cast<float2*>(smem_raw + L::twin); }
  static __device__ __forceinline__ float2* rin() { return reinterpret_cast<float2*>(smem_raw + L::rin); }
  static __device__ __forceinline__ float2* rout() { return reinterpret_cast<float2*>(smem_raw + L::rout); }
  static __device__ __forceinline__ float2* ws() { return reinterpret_cast<float2*>(smem_raw + L::ws); }
  static __device__ __forceinline__ float2** colptr() { return reinterpret_cast<float2**>(smem_raw + L::colptr); }
  static __device__ __forceinline__ float* red() { return reinterpret_cast<float*>(smem_raw + L::red); }
  static __device__ __forceinline__ float* sigpart() { return reinterpret_cast<float*>(smem_raw + L::sigpart); }
  static __device__ __forceinline__ int* slotb() { return reinterpret_cast<int*>(smem_raw + L::slotb); }
};

template <int F, int NC>
constexpr size_t smem_bytes() { return Lay<F, NC>::total; }

size_t correlate_smem_bytes(const Geometry& g) {
  if (g.F == 4096) {
    if (g.NC == 4) return smem_bytes<4096, 4>();
    if (g.NC == 2) return smem_bytes<4096, 2>();
    return smem_bytes<4096, 1>();
  }
  if (g.F == 2048) return smem_bytes<2048, 1>();
  if (g.F == 1024) return smem_bytes<1024, 1>();
  return smem_bytes<512, 1>();
}

// Column b held by slot c of the CTA with cluster rank `rank`.
__device__ __forceinline__ int slot_column(const Geometry& g, int rank, int c) {
  if (g.S == 1) return 0;
  const int ug = rank * g.UPC + (c >> 1);
  const int second = c & 1;
  if (ug == 0) return second ? g.S / 2 : 0;
  return second ? g.S - ug : ug;
}

// Owner CTA rank and slot of column b.
__device__ __forceinline__ void column_home(const Geometry& g, int b, int* owner, int* slot) {
  if (g.S == 1) {
    *owner = 0;
    *slot = 0;
    return;
  }
  int unit, second;
  if (b == 0) {
    unit = 0; second = 0;
  } else if (b == g.S / 2) {
    unit = 0; second = 1;
  } else if (b < g.S / 2) {
    unit = b; second = 0;
  } else {
    unit = g.S - b; second = 1;
  }
  *owner = unit / g.UPC;
  *slot = 2 * (unit % g.UPC) + second;
}

// Load the per-N twiddle tables into shared memory and resolve the
// (possibly remote) address of every column.
template <int F, int NC>
__device__ void setup_tables(const PlanDev& p, int rank, bool map_columns) {
  using SM = Smem<F, NC>;
  const Geometry& g = p.g;
  const int t = threadIdx.x;
  for (int i = t; i < F; i += kThreads) SM::tw3()[i] = p.tw3[i];
  for (int i = t; i < 16 * (F / 256); i += kThreads) SM::tw2()[i] = p.tw2[i];
  for (int i = t; i < NC * 256; i += kThreads) {
    const int c = i >> 8, j = i & 255;
    const int b = slot_column(g, rank, c);
    SM::twin()[i] = p.wH[b * j];
  }
  for (int i = t; i < NC * 16; i += kThreads) {
    const int c = i >> 4, r = i & 15;
    const int b = slot_column(g, rank, c);
    SM::rin()[i] = r < F / 256 ? p.wR0S[b * r] : make_float2(1.f, 0.f);
    SM::rout()[i] = cconj(p.w16S[b * r]);
  }
  if (t < 16) SM::ws()[t] = t < g.S ? p.wS[t] : make_float2(1.f, 0.f);
  if (t < NC) SM::slotb()[t] = slot_column(g, rank, t);
  if (map_columns && t < g.S) {
    int owner, slot;
    column_home(g, t, &owner, &slot);
    cg::cluster_group cl = cg::this_cluster();
    float2* base = cl.map_shared_rank(SM::cols(), (unsigned)owner);
    SM::colptr()[t] = base + slot * col_stride<F>();
  }
}

// First forward pass (radix R0 = F/256, Ns = 1) fused with the load of
// u_b[m1] = wH^(b m1) sum_{m2} z[m1 + F m2] wS^(b m2) from global memory.
// src holds nz complex samples z[m] (interleaved floats).
template <int F, int NC>
__device__ __forceinline__ void fwd_first_pass(int S, const float* __restrict__ src, int nz,
                                               int nfold) {
  using SM = Smem<F, NC>;
  constexpr int R0 = F / 256;
  constexpr int total = NC * 256;
  const float2* z = reinterpret_cast<const float2*>(src);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int idx = threadIdx.x + i * kThreads;
    if (idx < total) {
      const int c = idx >> 8, j = idx & 255;
      float2 v[R0];
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        const int m1 = j + r * 256;
        float2 acc = make_float2(0.f, 0.f);
        if (m1 < nz) acc = __ldg(z + m1);
        if (nfold > 1) {
          const int b = SM::slotb()[c];
          for (int m2 = 1; m2 < nfold; ++m2) {
            const int m = m1 + F * m2;
            if (m < nz) acc = cadd(acc, cmul(__ldg(z + m), SM::ws()[(b * m2) & (S - 1)]));
          }
        }
        v[r] = acc;
      }
      if (S > 1) {
        const float2 tj = SM::twin()[c * 256 + j];
#pragma unroll
        for (int r = 0; r < R0; ++r) v[r] = cmul(cmul(v[r], tj), SM::rin()[c * 16 + r]);
      }
      dft<R0, false>(v);
      float2* col = SM::col(c);
#pragma unroll
      for (int r = 0; r < R0; ++r) col[pad(j * R0 + r)] = v[r];
    }
  }
  __syncthreads();
}

// Last inverse pass (radix 16, Ns = F/16) fused with the output twiddle
// T_b[n1] = wH^(-b n1) x[n1], n1 = k + r F/16, factored as
// conj(wH^(b k)) * w(16 S)^(-b r).
template <int F, int NC>
__device__ __forceinline__ void inv_last_pass(int S) {
  using SM = Smem<F, NC>;
  constexpr int NB = F / 16;
  constexpr int Ns = F / 16;
  constexpr int total = NC * NB;
  constexpr int rounds = (total + kThreads - 1) / kThreads;
#pragma unroll
  for (int i = 0; i < rounds; ++i) {
    const int idx = threadIdx.x + i * kThreads;
    const bool act = idx < total;
    const int c = idx / NB, j = idx - c * NB;
    float2 v[16];
    if (act) {
      const float2* col = SM::col(c);
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = col[pad(j + r * NB)];
#pragma unroll
      for (int r = 1; r < 16; ++r) v[r] = cmulc(v[r], SM::tw3()[r * Ns + j]);
      dft<16, true>(v);
      if (S > 1) {
        const float2 tk = SM::twin()[c * 256 + j];
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = cmul(cmulc(v[r], tk), SM::rout()[c * 16 + r]);
      }
    }
    __syncthreads();
    if (act) {
      float2* col = SM::col(c);
#pragma unroll
      for (int r = 0; r < 16; ++r) col[pad(j + r * Ns)] = v[r];
    }
  }
  __syncthreads();
}

template <int F, int NC>
__device__ __forceinline__ void forward_columns(int S, const float* src, int nz, int nfold) {
  using SM = Smem<F, NC>;
  constexpr int R0 = F / 256;
  fwd_first_pass<F, NC>(S, src, nz, nfold);
  stockham_pass<F, 16, false>(SM::cols(), NC, R0, SM::tw2());
  stockham_pass<F, 16, false>(SM::cols(), NC, 16 * R0, SM::tw3());
}

template <int F, int NC>
__device__ __forceinline__ void inverse_columns(int S) {
  using SM = Smem<F, NC>;
  constexpr int R0 = F / 256;
  stockham_pass<F, R0, true>(SM::cols(), NC, 1, nullptr);
  stockham_pass<F, 16, true>(SM::cols(), NC, R0, SM::tw2());
  inv_last_pass<F, NC>(S);
}

// Enumerate the bin pairs (j, H-j) held by this CTA.  Unit 0 holds column 0
// (pairs a <-> (F-a) mod F, with a = 0 and a = F/2 paired with themselves)
// and column S/2 (pairs a <-> F-1-a); unit i holds columns i and S-i (pairs
// (i, a) <-> (S-i, F-1-a)).
struct PairItem {
  int b, a, bp, ap, sj, sp;  // columns, rows, local slots
};

template <int F>
__device__ __forceinline__ int unit_items(int S, int ug) {
  return ug == 0 ? (S >= 2 ? F + 1 : F / 2 + 1) : F;
}

template <int F>
__device__ __forceinline__ PairItem pair_item(int S, int ug, int ui, int it) {
  PairItem p;
  if (ug == 0) {
    if (it <= F / 2) {
      p.b = 0; p.a = it; p.bp = 0; p.ap = (F - it) & (F - 1);
      p.sj = p.sp = 2 * ui;
    } else {
      p.b = S / 2; p.a = it - (F / 2 + 1); p.bp = p.b; p.ap = F - 1 - p.a;
      p.sj = p.sp = 2 * ui + 1;
    }
  } else {
    p.b = ug; p.a = it; p.bp = S - ug; p.ap = F - 1 - it;
    p.sj = 2 * ui; p.sp = 2 * ui + 1;
  }
  return p;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// S1: segment spectrum D and product coefficients A, B
// ---------------------------------------------------------------------------
template <int F, int NC>
__global__ void __launch_bounds__(kThreads, 1)
segment_kernel(PlanDev p, const float* __restrict__ y, float2* __restrict__ D,
               float4* __restrict__ AB) {
  using SM = Smem<F, NC>;
  const Geometry g = p.g;
  const int S = g.S;
  const int rank = blockIdx.x;
  constexpr int UPC = NC == 1 ? 1 : NC / 2;
  setup_tables<F, NC>(p, rank, false);
  __syncthreads();
  forward_columns<F, NC>(S, y, g.H, S);

  for (int ui = 0; ui < UPC; ++ui) {
    const int ug = rank * UPC + ui;
    const int count = unit_items<F>(S, ug);
    for (int it = threadIdx.x; it < count; it += kThreads) {
      const PairItem q = pair_item<F>(S, ug, ui, it);
      const float2 zj = SM::col(q.sj)[pad(q.a)];
      const float2 zp = SM::col(q.sp)[pad(q.ap)];
      const int j = S * q.a + q.b;
      const int jp = S * q.ap + q.bp;
      const bool self = (j == jp);
      // D_j = (Zj + conj Zp)/2 - (i/2) wN^j (Zj - conj Zp)
      const float2 wj = p.wN[j];
      const float2 sj = cadd(zj, cconj(zp)), dj = csub(zj, cconj(zp));
      const float2 dd = cmul(wj, dj);
      const float2 Dj = make_float2(0.5f * (sj.x + dd.y), 0.5f * (sj.y - dd.x));
      float2 Djp = Dj;
      if (!self) {
        const float2 wp = p.wN[jp];
        const float2 sp = cadd(zp, cconj(zj)), dp = csub(zp, cconj(zj));
        const float2 de = cmul(wp, dp);
        Djp = make_float2(0.5f * (sp.x + de.y), 0.5f * (sp.y - de.x));
      }
      const float2 DH = make_float2(zj.x - zj.y, 0.f);  // D_{N/2}, used when j == 0
      // conj D_{H-j}: for j = 0 it is the Nyquist bin, otherwise conj D_jp
      const float2 cHj = (j == 0) ? DH : cconj(Djp);
      const float2 cHjp = cconj(Dj);
      auto coeffs = [](float2 w, float2 Dx, float2 cH) {
        // g = (1 + i conj w)/2, d = (1 - i conj w)/2 with i conj(w) = (w.y, w.x)
        const float2 gg = make_float2(0.5f * (1.f + w.y), 0.5f * w.x);
        const float2 de = make_float2(0.5f * (1.f - w.y), -0.5f * w.x);
        const float2 A = cadd(cmul(cmul(gg, gg), Dx), cmul(cmul(de, de), cH));
        const float2 B = cmul(cmul(gg, de), cadd(Dx, cH));
        return make_float4(A.x, A.y, B.x, B.y);
      };
      AB[q.b * F + q.a] = coeffs(wj, Dj, cHj);
      D[j] = Dj;
      if (!self) {
        AB[q.bp * F + q.ap] = coeffs(p.wN[jp], Djp, cHjp);
        D[jp] = Djp;
      }
      if (j == 0) D[g.H] = DH;
    }
  }
}

// ---------------------------------------------------------------------------
// S2-S6: template spectrum, product, sigma, inverse FFT, threshold, compaction
// ---------------------------------------------------------------------------
template <int F, int NC, int SS>
__device__ __forceinline__ void combine_and_emit(int C, int H, int rank, float thr,
                                                 uint32_t tmpl, int64_t krow,
                                                 const CorrelateArgs& a) {
  using SM = Smem<F, NC>;
  const int per = F / C;
  const int iters = per / kThreads;
  const int lane = threadIdx.x & 31;
  const float invH = 1.0f / (float)H;
  float2* const* colptr = SM::colptr();
  for (int it = 0; it < iters; ++it) {
    const int n1 = rank * per + it * kThreads + threadIdx.x;
    float2 t[SS];
#pragma unroll
    for (int b = 0; b < SS; ++b) t[b] = colptr[b][pad(n1)];
    dft<SS, true>(t);
    uint32_t mask = 0;
#pragma unroll
    for (int n2 = 0; n2 < SS; ++n2) {
      t[n2] = cscale(t[n2], invH);
      mask |= (fabsf(t[n2].x) > thr ? 1u : 0u) << (2 * n2);
      mask |= (fabsf(t[n2].y) > thr ? 1u : 0u) << (2 * n2 + 1);
    }
    if (a.dump) {
      float2* row = reinterpret_cast<float2*>(a.dump) + krow * (int64_t)H;
#pragma unroll
      for (int n2 = 0; n2 < SS; ++n2) row[n1 + F * n2] = t[n2];
    }
    if (__any_sync(0xffffffffu, mask != 0u)) {
      const int cnt = __popc(mask);
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      unsigned long long base = 0;
      if (lane == 31) base = atomicAdd(a.counter, (unsigned long long)total);
      base = __shfl_sync(0xffffffffu, base, 31);
      unsigned long long pos = base + (unsigned long long)(incl - cnt);
#pragma unroll
      for (int n2 = 0; n2 < SS; ++n2) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if ((mask >> (2 * n2 + e)) & 1u) {
            if (pos < a.cap) {
              bege_tail* r = a.recs + pos;
              r->tmpl = tmpl;
              r->lag = (uint32_t)(2 * (n1 + F * n2) + e);
              r->value = e ? t[n2].y : t[n2].x;
            }
            ++pos;
          }
        }
      }
    }
  }
}

template <int F, int NC>
__global__ void __launch_bounds__(kThreads, 1) correlate_kernel(PlanDev p, CorrelateArgs a) {
  using SM = Smem<F, NC>;
  constexpr int UPC = NC == 1 ? 1 : NC / 2;
  cg::cluster_group cluster = cg::this_cluster();
  const int S = p.g.S;
  const int C = S >= 2 * NC ? S / NC : 1;
  const int N = p.g.N, H = p.g.H;
  const int rank = (int)cluster.block_rank();
  setup_tables<F, NC>(p, rank, true);
  __syncthreads();

  const int cid = blockIdx.x / C;
  const int ncl = gridDim.x / C;
  const int nz = (int)(a.Lp / 2);
  const int nfold = (nz + F - 1) / F;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  for (int64_t k = a.k0 + cid; k < a.k1; k += ncl) {
    // S2: template spectrum (column FFTs of the packed, twiddled template)
    forward_columns<F, NC>(S, a.bank + k * a.Lp, nz, nfold);

    // S3 + S4: Y = conj(Z) A + Z' B over this CTA's bin pairs, sum |Y|^2
    float acc = 0.f;
#pragma unroll
    for (int ui = 0; ui < UPC; ++ui) {
      const int ug = rank * UPC + ui;
      const int count = unit_items<F>(S, ug);
      for (int it = threadIdx.x; it < count; it += kThreads) {
        const PairItem q = pair_item<F>(S, ug, ui, it);
        float2* cj = SM::col(q.sj) + pad(q.a);
        float2* cp = SM::col(q.sp) + pad(q.ap);
        const float2 zj = *cj, zp = *cp;
        const float4 abj = __ldcg(a.AB + q.b * F + q.a);
        const float2 yj = cadd(cconjmul(zj, make_float2(abj.x, abj.y)),
                               cmul(zp, make_float2(abj.z, abj.w)));
        acc = fmaf(yj.x, yj.x, fmaf(yj.y, yj.y, acc));
        if (cj != cp) {
          const float4 abp = __ldcg(a.AB + q.bp * F + q.ap);
          const float2 yp = cadd(cconjmul(zp, make_float2(abp.x, abp.y)),
                                 cmul(zj, make_float2(abp.z, abp.w)));
          acc = fmaf(yp.x, yp.x, fmaf(yp.y, yp.y, acc));
          *cp = yp;
        }
        *cj = yj;
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) SM::red()[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float s = 0.f;
      for (int w = 0; w < kThreads / 32; ++w) s += SM::red()[w];
      *SM::sigpart() = s;
    }

    // S5: inverse column FFTs (the first pass reads after the barrier above)
    inverse_columns<F, NC>(S);

    cluster.sync();  // every column and every sigma partial of the cluster is ready

    float tot = 0.f;
    for (int q = 0; q < C; ++q) tot += *cluster.map_shared_rank(SM::sigpart(), (unsigned)q);
    const float sigma = sqrtf(2.0f * tot) / (float)N;
    const float thr = a.kappa * sigma;
    const int64_t krow = k - a.k0;
    if (rank == 0 && threadIdx.x == 0) a.sigma[krow] = sigma;

    // S6: S-point combine, threshold, warp-ballot compaction
    if constexpr (NC == 1) {
      combine_and_emit<F, NC, 1>(C, H, rank, thr, (uint32_t)k, krow, a);
    } else if constexpr (NC == 2) {
      combine_and_emit<F, NC, 2>(C, H, rank, thr, (uint32_t)k, krow, a);
    } else {
      switch (S) {
        case 4: combine_and_emit<F, NC, 4>(C, H, rank, thr, (uint32_t)k, krow, a); break;
        case 8: combine_and_emit<F, NC, 8>(C, H, rank, thr, (uint32_t)k, krow, a); break;
        default: combine_and_emit<F, NC, 16>(C, H, rank, thr, (uint32_t)k, krow, a); break;
      }
    }

    cluster.sync();  // remote reads done before the columns are overwritten
  }
}

// ---------------------------------------------------------------------------
// Bank synthesis: w[m] = T(m) sin(2 pi phase(m)), unit L2 norm
// ---------------------------------------------------------------------------
__device__ __forceinline__ double chirp_sample(unsigned long long alpha, unsigned long long beta,
                                               int64_t m, int64_t L, int width, double denom) {
  const unsigned long long um = (unsigned long long)m;
  // phase in cycles * 2^64, exact modulo one cycle
  const unsigned long long ph = alpha * um + beta * (um * um);
  const double c = (double)(long long)ph * 0x1p-64;  // in [-1/2, 1/2)
  const double s = sinpi(2.0 * c);
  const int64_t mm = m < L - 1 - m ? m : L - 1 - m;
  double t = 1.0;
  if (mm <= width) t = 0.5 * (1.0 - cospi(2.0 * (double)mm / denom));
  return t * s;
}

__global__ void __launch_bounds__(256) bank_chirp_kernel(const unsigned long long* __restrict__ ab,
                                                         int64_t L, int64_t Lp, double frac,
                                                         float* __restrict__ bank) {
  __shared__ double red[8];
  const int64_t k = blockIdx.x;
  const unsigned long long alpha = ab[2 * k], beta = ab[2 * k + 1];
  const int width = (frac > 0.0 && L >= 2) ? (int)floor(frac * (double)(L - 1) / 2.0) : -1;
  const double denom = frac * (double)(L - 1);
  double acc = 0.0;
  for (int64_t m = threadIdx.x; m < L; m += blockDim.x) {
    const double v = chirp_sample(alpha, beta, m, L, width, denom);
    acc = fma(v, v, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  double norm = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) norm += red[w];
  const double scale = norm > 0.0 ? 1.0 / sqrt(norm) : 0.0;
  float* row = bank + k * Lp;
  for (int64_t m = threadIdx.x; m < Lp; m += blockDim.x)
    row[m] = m < L ? (float)(chirp_sample(alpha, beta, m, L, width, denom) * scale) : 0.f;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename K>
static cudaError_t ensure_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int F, int NC>
static cudaError_t launch_segment_t(const PlanDev& p, const float* y, float2* D, float4* AB,
                                    cudaStream_t s) {
  constexpr size_t smem = smem_bytes<F, NC>();
  cudaError_t e = ensure_smem(segment_kernel<F, NC>, smem);
  if (e != cudaSuccess) return e;
  segment_kernel<F, NC><<<p.g.C, kThreads, smem, s>>>(p, y, D, AB);
  return cudaGetLastError();
}

cudaError_t launch_segment(const PlanDev& p, const float* y, float2* D, float4* AB,
                           cudaStream_t s) {
  const Geometry& g = p.g;
  if (g.F == 4096) {
    if (g.NC == 4) return launch_segment_t<4096, 4>(p, y, D, AB, s);
    if (g.NC == 2) return launch_segment_t<4096, 2>(p, y, D, AB, s);
    return launch_segment_t<4096, 1>(p, y, D, AB, s);
  }
  if (g.F == 2048) return launch_segment_t<2048, 1>(p, y, D, AB, s);
  if (g.F == 1024) return launch_segment_t<1024, 1>(p, y, D, AB, s);
  if (g.F == 512) return launch_segment_t<512, 1>(p, y, D, AB, s);
  return cudaErrorInvalidValue;
}

template <int F, int NC>
static cudaError_t launch_correlate_t(const PlanDev& p, const CorrelateArgs& a, cudaStream_t s) {
  constexpr size_t smem = smem_bytes<F, NC>();
  cudaError_t e = ensure_smem(correlate_kernel<F, NC>, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)p.g.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  cfg.gridDim = dim3((unsigned)(sms / p.g.C * p.g.C), 1, 1);
  int max_clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&max_clusters, correlate_kernel<F, NC>, &cfg);
  if (e != cudaSuccess) return e;
  if (max_clusters < 1) return cudaErrorInvalidConfiguration;
  int64_t want = a.k1 - a.k0;
  if (a.max_clusters > 0 && want > a.max_clusters) want = a.max_clusters;
  if (want > max_clusters) want = max_clusters;
  cfg.gridDim = dim3((unsigned)(want * p.g.C), 1, 1);
  return cudaLaunchKernelEx(&cfg, correlate_kernel<F, NC>, p, a);
}

cudaError_t launch_correlate(const PlanDev& p, const CorrelateArgs& a, cudaStream_t s) {
  if (a.k1 <= a.k0) return cudaSuccess;
  const Geometry& g = p.g;
  if (g.F == 4096) {
    if (g.NC == 4) return launch_correlate_t<4096, 4>(p, a, s);
    if (g.NC == 2) return launch_correlate_t<4096, 2>(p, a, s);
    return launch_correlate_t<4096, 1>(p, a, s);
  }
  if (g.F == 2048) return launch_correlate_t<2048, 1>(p, a, s);
  if (g.F == 1024) return launch_correlate_t<1024, 1>(p, a, s);
  if (g.F == 512) return launch_correlate_t<512, 1>(p, a, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_bank_chirp(const unsigned long long* alpha_beta, int64_t count, int64_t L,
                              int64_t Lp, double taper_frac, float* bank, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  bank_chirp_kernel<<<(unsigned)count, 256, 0, s>>>(alpha_beta, L, Lp, taper_frac, bank);
  return cudaGetLastError();
}

}  // namespace bege
