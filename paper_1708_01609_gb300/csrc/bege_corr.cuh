// Kernels of the matched-filter hot path, templated on the geometry.
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
// a template of L <= 2F samples has z = 0 beyond F, so only m2 = 0 remains
// (and with L <= F the upper half of u_b is zero as well).  Inverse, with
// n = n1 + F n2,
//     yo[n1 + F n2] = (1/H) sum_b wS^(-b n2) T_b[n1],
//     T_b[n1] = wH^(-b n1) IFFT_F(Y_{S.+b})[n1].
// Column b pairs with column S-b (bins j and H-j); columns {0, S/2} and
// {i, S-i} form units.  A CTA owns whole units (NC columns); the C = S/NC
// CTAs of a thread-block cluster hold all S columns and read each other's
// columns through distributed shared memory only in the final S-point
// combine.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bege_fft.cuh"
#include "bege_internal.h"

namespace bege {

namespace cg = cooperative_groups;

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
  static constexpr size_t sigall = sigpart + align16(4);
  static constexpr size_t total = sigall + align16(16 * 4);
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
  static __device__ __forceinline__ float* sigall() { return reinterpret_cast<float*>(smem_raw + L::sigall); }
};

// Column ownership for S >= 2 columns split over S/NC CTAs, S given at run
// time: unit u (u < S/2) holds columns u and S-u, unit 0 columns 0 and S/2;
// a CTA holds NC/2 consecutive units.
template <int NC>
__device__ __forceinline__ int slot_column_rt(int S, int rank, int c) {
  const int ug = rank * (NC / 2) + (c >> 1);
  const int second = c & 1;
  if (ug == 0) return second ? S / 2 : 0;
  return second ? S - ug : ug;
}
template <int NC>
__device__ __forceinline__ void home_rt(int S, int b, int* owner, int* slot) {
  int unit, second;
  if (b == 0) {
    unit = 0; second = 0;
  } else if (b == S / 2) {
    unit = 0; second = 1;
  } else if (b < S / 2) {
    unit = b; second = 0;
  } else {
    unit = S - b; second = 1;
  }
  *owner = unit / (NC / 2);
  *slot = 2 * (unit % (NC / 2)) + second;
}

// Column ownership for S columns split over C = S/NC CTAs.
template <int S, int NC>
struct ColMap {
  static_assert(S == 1 ? NC == 1 : (NC % 2 == 0 && S % NC == 0), "column split");
  static constexpr int C = S == 1 ? 1 : S / NC;
  static constexpr int UPC = S == 1 ? 1 : NC / 2;
  // column b held by local slot c of the CTA with cluster rank `rank`
  static __device__ __forceinline__ int slot_column(int rank, int c) {
    if constexpr (S == 1)
      return 0;
    else
      return slot_column_rt<NC>(S, rank, c);
  }
  // owner rank and local slot of column b
  static __device__ __forceinline__ void home(int b, int* owner, int* slot) {
    if constexpr (S == 1) {
      *owner = 0;
      *slot = 0;
    } else {
      home_rt<NC>(S, b, owner, slot);
    }
  }
};

// The functions below take the column count S as a template argument; S = 0
// means "given at run time" (argument s_rt, S >= 2), which lets one kernel
// body serve every segment length with the same arithmetic.
template <int S, int NC>
__device__ __forceinline__ int slot_col(int s_rt, int rank, int c) {
  if constexpr (S == 1)
    return 0;
  else
    return slot_column_rt<NC>(S ? S : s_rt, rank, c);
}

// Twiddle tables that depend on F only (the Stockham passes).
template <int F, int NC, int T>
__device__ void setup_common(const PlanDev& p) {
  using SM = Smem<F, NC>;
  for (int i = threadIdx.x; i < F; i += T) SM::tw3()[i] = p.tw3[i];
  for (int i = threadIdx.x; i < 16 * (F / 256); i += T) SM::tw2()[i] = p.tw2[i];
}

// Column twiddles of this CTA's slots (rank `grank` within its group of
// C = S/NC CTAs) and the (possibly remote) address of every column of the
// group, whose first CTA has cluster rank `gbase`.
template <int F, int S, int NC, int T>
__device__ void setup_columns(const PlanDev& p, int grank, int gbase, bool map_columns,
                              int s_rt = S) {
  using SM = Smem<F, NC>;
  const int Sv = S ? S : s_rt;
  const int t = threadIdx.x;
  for (int i = t; i < NC * 256; i += T) {
    const int c = i >> 8, j = i & 255;
    SM::twin()[i] = p.wH[slot_col<S, NC>(Sv, grank, c) * j];
  }
  for (int i = t; i < NC * 16; i += T) {
    const int c = i >> 4, r = i & 15;
    const int b = slot_col<S, NC>(Sv, grank, c);
    SM::rin()[i] = r < F / 256 ? p.wR0S[b * r] : make_float2(1.f, 0.f);
    SM::rout()[i] = cconj(p.w16S[b * r]);
  }
  if (t < 16) SM::ws()[t] = t < Sv ? p.wS[t] : make_float2(1.f, 0.f);
  if (map_columns && t < Sv) {
    int owner, slot;
    if constexpr (S == 1) {
      owner = 0;
      slot = 0;
    } else {
      home_rt<NC>(Sv, t, &owner, &slot);
    }
    cg::cluster_group cl = cg::this_cluster();
    float2* base = cl.map_shared_rank(SM::cols(), (unsigned)(gbase + owner));
    SM::colptr()[t] = base + slot * col_stride<F>();
  }
}

// First forward pass (radix R0 = F/256, Ns = 1) fused with the load of
// u_b[m1] = wH^(b m1) sum_{m2} z[m1 + F m2] wS^(b m2) from global memory.
// src holds nz complex samples z[m] (interleaved floats).  HALFZ: nz <= F/2
// and the upper half of every radix-16 input vector is zero.
template <int F, int S, int NC, int T, bool HALFZ>
__device__ __forceinline__ void fwd_first_pass(int rank, const float* __restrict__ src, int nz,
                                               int nfold, int s_rt = S) {
  using SM = Smem<F, NC>;
  const int Sv = S ? S : s_rt;
  constexpr int R0 = F / 256;
  constexpr int RL = HALFZ ? R0 / 2 : R0;  // inputs that can be non-zero
  constexpr int total = NC * 256;
  const float2* z = reinterpret_cast<const float2*>(src);
#pragma unroll
  for (int i = 0; i < (total + T - 1) / T; ++i) {
    const int idx = threadIdx.x + i * T;
    if ((total % T == 0) || idx < total) {
      const int c = idx >> 8, j = idx & 255;
      float2 v[R0];
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        const int m1 = j + r * 256;
        float2 acc = make_float2(0.f, 0.f);
        if (r < RL) {
          if (m1 < nz) acc = __ldg(z + m1);
          if (!HALFZ && nfold > 1) {
            const int b = slot_col<S, NC>(Sv, rank, c);
            for (int m2 = 1; m2 < nfold; ++m2) {
              const int m = m1 + F * m2;
              if (m < nz) acc = cadd(acc, cmul(__ldg(z + m), SM::ws()[(b * m2) & (Sv - 1)]));
            }
          }
        }
        v[r] = acc;
      }
      if constexpr (S != 1) {
        const float2 tj = SM::twin()[c * 256 + j];
        const float2* rin = SM::rin() + c * 16;
#pragma unroll
        for (int r = 0; r < RL; ++r) v[r] = cmul(cmul(v[r], tj), rin[r]);
      }
      dft<R0, false, HALFZ>(v);
      float2* col = SM::col(c) + pad(j * R0);
#pragma unroll
      for (int r = 0; r < R0; ++r) col[r] = v[r];  // R0 <= 16 consecutive: one pad group
    }
  }
  __syncthreads();
}

// Last inverse pass (radix 16, Ns = F/16) fused with the output twiddle
// T_b[n1] = wH^(-b n1) x[n1], n1 = k + r F/16, factored as
// conj(wH^(b k)) * w(16 S)^(-b r).
template <int F, int S, int NC, int T, bool TRAIL = true>
__device__ __forceinline__ void inv_last_pass() {
  using SM = Smem<F, NC>;
  constexpr int NB = F / 16;
  constexpr int Ns = F / 16;
  constexpr int total = NC * NB;
  constexpr int rounds = (total + T - 1) / T;
  constexpr int step = Ns + Ns / 16;
#pragma unroll
  for (int i = 0; i < rounds; ++i) {
    const int idx = threadIdx.x + i * T;
    const bool act = (total % T == 0) || idx < total;
    const int c = idx / NB, j = idx - c * NB;
    float2 v[16];
    if (act) {
      const float2* col = SM::col(c) + pad(j);
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = col[r * step];
      const float2* t3 = SM::tw3() + j;
#pragma unroll
      for (int r = 1; r < 16; ++r) v[r] = cmulc(v[r], t3[r * Ns]);
      dft<16, true>(v);
      if constexpr (S != 1) {
        const float2 tk = SM::twin()[c * 256 + j];
        const float2* ro = SM::rout() + c * 16;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = cmul(cmulc(v[r], tk), ro[r]);
      }
    }
    __syncthreads();
    if (act) {
      float2* col = SM::col(c) + pad(j);
#pragma unroll
      for (int r = 0; r < 16; ++r) col[r * step] = v[r];
    }
  }
  if constexpr (TRAIL) __syncthreads();
}

template <int F, int S, int NC, int T, bool HALFZ>
__device__ __forceinline__ void forward_columns(int rank, const float* src, int nz, int nfold) {
  using SM = Smem<F, NC>;
  constexpr int R0 = F / 256;
  fwd_first_pass<F, S, NC, T, HALFZ>(rank, src, nz, nfold);
  stockham_pass<F, NC, T, 16, R0, false>(SM::cols(), SM::tw2());
  stockham_pass<F, NC, T, 16, 16 * R0, false>(SM::cols(), SM::tw3());
}

template <int F, int S, int NC, int T>
__device__ __forceinline__ void inverse_columns() {
  using SM = Smem<F, NC>;
  constexpr int R0 = F / 256;
  stockham_pass<F, NC, T, R0, 1, true>(SM::cols(), nullptr);
  stockham_pass<F, NC, T, 16, R0, true>(SM::cols(), SM::tw2());
  inv_last_pass<F, S, NC, T>();
}

// The bin pairs (j, H-j) held by a unit.  Unit 0 holds column 0 (pairs
// a <-> (F-a) mod F, with a = 0 and a = F/2 paired with themselves) and
// column S/2 (pairs a <-> F-1-a); unit i holds columns i and S-i (pairs
// (i, a) <-> (S-i, F-1-a)).
struct PairItem {
  int b, a, bp, ap, sj, sp;  // columns, rows, local slots
};

template <int F, int S>
__device__ __forceinline__ int unit_items(int ug) {
  return ug == 0 ? (S >= 2 ? F + 1 : F / 2 + 1) : F;
}

template <int F, int S>
__device__ __forceinline__ PairItem pair_item(int ug, int ui, int it) {
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

// Y = conj(x) A + y B with ab = {A, B}: the spectral product of Eq. 3S in
// the packed form.  (Written as two chains of fused multiply-adds it needs
// two instructions fewer per value, but the longer chains make the fused
// middle stage spill.)
__device__ __forceinline__ float2 packed_product(float2 x, float2 y, float4 ab) {
  const float2 xa = make_float2(fmaf(x.x, ab.x, x.y * ab.y), fmaf(x.x, ab.y, -x.y * ab.x));
  return cadd(xa, cmul(y, make_float2(ab.z, ab.w)));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Fused middle of the pipeline for F = 4096 (radix 16 x 16 x 16): the last
// forward pass, the spectral product with the Parseval sum, and the first
// inverse pass, in registers.
//
// Forward pass 3 (Ns = 256) reads and writes the rows j + 256 r of its
// butterfly j, and inverse pass 1 (Ns = 1) reads the same rows, so one thread
// can carry a butterfly from the forward FFT into the inverse FFT.  The bin
// (b, j + 256 r) pairs with (S-b, (255-j) + 256 (15-r)) (column 0: with
// (0, (256-j) + 256 (15-r)), column S/2: with (S/2, (255-j) + 256 (15-r))),
// i.e. with row 15-r of the mirror butterfly, so a thread that holds a
// butterfly and its mirror forms every Y of both.  Items (256 per unit):
//   generic unit ug:  (slot 2ui, j) with (slot 2ui+1, 255-j),   j < 256
//   unit 0, it < 128: column 0, (j, 256-j); it = 0 holds the two
//                     self-mirrored butterflies 0 and 128
//   unit 0, it >= 128: column S/2, (j, 255-j), j = it - 128
// Returns this thread's sum of |Y|^2; ends with the stores of inverse pass 1
// (callers synchronise before reading the columns).
// ---------------------------------------------------------------------------
//
// MULTI (several segments against one template): the forward half's output
// Z (za, zb) is kept in `scratch` (this thread's 32 values, stride T; none
// for a single segment); with `reload` the forward half is skipped and Z is
// read back from there.
template <int S, int NC, int T, bool MULTI = false>
__device__ __forceinline__ float fused_mid(int rank, const float4* __restrict__ AB,
                                           float* red_warp, int s_rt = S,
                                           float2* __restrict__ scratch = nullptr,
                                           bool reload = false) {
  constexpr int F = 4096;
  using SM = Smem<F, NC>;
  constexpr int UPC = S == 1 ? 1 : NC / 2;
  constexpr int items = S == 1 ? 128 : 256;  // per unit
  const int Sv = S ? S : s_rt;
  static_assert(T >= items * UPC, "one item per thread");
  constexpr int step = 256 + 16;             // padded distance of rows r -> r + 1
  const int t = threadIdx.x;
  const bool act = t < items * UPC;
  const int ui = t / items, it = t - ui * items;
  const int ug = rank * UPC + ui;
  // columns and butterflies of the item
  int sa, sb, ja, jb, ba, bb;
  bool self0 = false;  // column 0, butterflies 0 and 128 (each its own mirror)
  if (ug == 0 && it < 128) {
    sa = sb = 2 * ui; ba = bb = 0;
    ja = it; jb = it == 0 ? 128 : 256 - it;
    self0 = (it == 0);
  } else if (ug == 0) {
    sa = sb = 2 * ui + 1; ba = bb = Sv / 2;
    ja = it - 128; jb = 255 - ja;
  } else {
    sa = 2 * ui; sb = 2 * ui + 1; ba = ug; bb = Sv - ug;
    ja = it; jb = 255 - it;
  }
  float2 za[16], zb[16];
  float acc = 0.f;
  if (act) {
    if (MULTI && reload) {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        za[r] = __ldcg(scratch + r * T + t);
        zb[r] = __ldcg(scratch + (16 + r) * T + t);
      }
    } else {
      const float2* pa = SM::col(sa) + pad(ja);
      const float2* pb = SM::col(sb) + pad(jb);
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        za[r] = pa[r * step];
        zb[r] = pb[r * step];
      }
      const float2* ta = SM::tw3() + ja;
      const float2* tb = SM::tw3() + jb;
#pragma unroll
      for (int r = 1; r < 16; ++r) {
        za[r] = cmul(za[r], ta[r * 256]);
        zb[r] = cmul(zb[r], tb[r * 256]);
      }
      dft<16, false>(za);
      dft<16, false>(zb);
      if (MULTI && scratch) {  // kept for the block's other segments
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          __stcg(scratch + r * T + t, za[r]);
          __stcg(scratch + (16 + r) * T + t, zb[r]);
        }
      }
    }
    const float4* aba = AB + ba * F + ja;
    const float4* abb = AB + bb * F + jb;
    if (!self0) {
      // za[r] (row ja + 256 r) pairs with zb[15 - r] (row jb + 256 (15 - r))
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const float4 p = __ldcg(aba + 256 * r);
        const float4 q = __ldcg(abb + 256 * (15 - r));
        const float2 x = za[r], y = zb[15 - r];
        const float2 ya = packed_product(x, y, p);
        const float2 yb = packed_product(y, x, q);
        acc = fmaf(ya.x, ya.x, fmaf(ya.y, ya.y, acc));
        acc = fmaf(yb.x, yb.x, fmaf(yb.y, yb.y, acc));
        za[r] = ya;
        zb[15 - r] = yb;
      }
    } else {
      // butterfly 0: rows 256 r pair with 256 ((16 - r) mod 16); r = 0, 8 self
      float2 ya[16], yb[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int rp = (16 - r) & 15;
        const float4 p = __ldcg(aba + 256 * r);
        ya[r] = packed_product(za[r], za[rp], p);
        acc = fmaf(ya[r].x, ya[r].x, fmaf(ya[r].y, ya[r].y, acc));
      }
      // butterfly 128: rows 128 + 256 r pair with 128 + 256 (15 - r)
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const float4 q = __ldcg(abb + 256 * r);
        yb[r] = packed_product(zb[r], zb[15 - r], q);
        acc = fmaf(yb[r].x, yb[r].x, fmaf(yb[r].y, yb[r].y, acc));
      }
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        za[r] = ya[r];
        zb[r] = yb[r];
      }
    }
    dft<16, true>(za);
    dft<16, true>(zb);
  }
  acc = warp_sum(acc);
  if ((t & 31) == 0) red_warp[t >> 5] = acc;
  __syncthreads();  // every load of the columns is done
  if (act) {
    // inverse pass 1 (Ns = 1): butterfly j writes rows 16 j + r
    float2* qa = SM::col(sa) + pad(16 * ja);
    float2* qb = SM::col(sb) + pad(16 * jb);
#pragma unroll
    for (int r = 0; r < 16; ++r) qa[r] = za[r];
#pragma unroll
    for (int r = 0; r < 16; ++r) qb[r] = zb[r];
  }
  return acc;
}

// fused_mid as a function of its own (see the interleaved kernel).
template <int S, int NC, int T>
__device__ __noinline__ float fused_mid_call(int rank, const float4* __restrict__ AB,
                                             float* red_warp) {
  return fused_mid<S, NC, T>(rank, AB, red_warp);
}

// ---------------------------------------------------------------------------
// S1: segment spectrum D and product coefficients A, B (grid: C CTAs)
// ---------------------------------------------------------------------------
template <int F, int S, int NC, int T>
__device__ __forceinline__ void segment_body(const PlanDev& p, int rank,
                                             const float* __restrict__ y,
                                             float2* __restrict__ D, float4* __restrict__ AB) {
  using SM = Smem<F, NC>;
  constexpr int UPC = ColMap<S, NC>::UPC;
  const int H = p.g.H;
  setup_common<F, NC, T>(p);
  setup_columns<F, S, NC, T>(p, rank, 0, false);
  __syncthreads();
  forward_columns<F, S, NC, T, false>(rank, y, H, S);

  for (int ui = 0; ui < UPC; ++ui) {
    const int ug = rank * UPC + ui;
    const int count = unit_items<F, S>(ug);
    for (int it = threadIdx.x; it < count; it += T) {
      const PairItem q = pair_item<F, S>(ug, ui, it);
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
      if (j == 0) D[H] = DH;
    }
  }
}

template <int F, int S, int NC, int T>
__global__ void __launch_bounds__(T, 1)
segment_kernel(PlanDev p, const float* __restrict__ y, float2* __restrict__ D,
               float4* __restrict__ AB) {
  segment_body<F, S, NC, T>(p, blockIdx.x, y, D, AB);
}

// ---------------------------------------------------------------------------
// S2-S6: template spectrum, product, sigma, inverse FFT, threshold, compaction
// ---------------------------------------------------------------------------
// Where one correlation's tails (and optional full dump) go.
struct TailOut {
  bege_tail* recs;
  uint64_t cap;
  unsigned long long* counter;
  float* dump;
  // optional per-lag maximum over the bank (Eq. Ak): one 64-bit word per
  // lag, (bits of rho/sigma) << 32 | ~template, raised with atomicMax
  unsigned long long* proj = nullptr;
  // optional upper end of a tail band (Sec. 5): keep |rho| < kappa_hi sigma
  // as well; 0 = no upper end
  float kappa_hi = 0.f;
  // optional overlap-save mask: tails only at lags n < lag_end (the lags
  // whose template window does not wrap); all N lags by default
  uint32_t lag_end = 0xffffffffu;
};

// EXT: the extended epilogue, the per-lag maximum a.proj, the band's upper
// end a.kappa_hi and the lag mask a.lag_end (compiled only into the kernels
// that serve bege_correlate_max, bege_correlate_band and bege_correlate_ex,
// so the others keep their code unchanged).  sigma: the template's sigma (thr = kappa sigma).
//
// IL: the columns are interleaved two per CTA (NC = 2); `colptr` then holds
// the C CTAs' row arrays (float4*, cast), CTA u holding columns u and S - u
// (CTA 0: 0 and S/2), and a row of both comes in one 16-byte load.
template <int F, int S, int NC, int T, bool EXT = false, bool IL = false>
__device__ __forceinline__ void combine_and_emit(float2* const* colptr, int H, int rank, float thr,
                                                 uint32_t tmpl, int64_t krow, const TailOut& a,
                                                 float sigma, int tix = threadIdx.x) {
  constexpr int C = ColMap<S, NC>::C;
  constexpr int per = F / C;
  static_assert(per % T == 0, "combine rounds");
  const int lane = threadIdx.x & 31;
  // rho = t / H with H a power of two: |t / H| > thr exactly when |t| > thr H,
  // so the unscaled values are tested and only the emitted ones are scaled
  const float invH = 1.0f / (float)H;
  const float thrH = thr * (float)H;
  // |t / H| < kappa_hi sigma exactly when |t| < kappa_hi sigma H (H a power of two)
  const float hiH = (EXT && a.kappa_hi > 0.f) ? a.kappa_hi * sigma * (float)H : INFINITY;
#pragma unroll 1
  for (int it = 0; it < per / T; ++it) {
    const int n1 = rank * per + it * T + tix;
    const int pn1 = pad(n1);
    float2 t[S];
    if constexpr (IL) {
      static_assert(NC == 2 && S >= 2, "interleaved columns: one unit per CTA");
#pragma unroll
      for (int u = 0; u < S / 2; ++u) {
        const float4 v = reinterpret_cast<const float4*>(colptr[u])[pn1];
        t[u] = make_float2(v.x, v.y);
        t[u == 0 ? S / 2 : S - u] = make_float2(v.z, v.w);
      }
    } else {
#pragma unroll
      for (int b = 0; b < S; ++b) t[b] = colptr[b][pn1];
    }
    dft<S, true>(t);
    float big = 0.f;
#pragma unroll
    for (int n2 = 0; n2 < S; ++n2) big = fmaxf(big, fmaxf(fabsf(t[n2].x), fabsf(t[n2].y)));
    if (a.dump) {
      float2* row = reinterpret_cast<float2*>(a.dump) + krow * (int64_t)H;
#pragma unroll
      for (int n2 = 0; n2 < S; ++n2) row[n1 + F * n2] = cscale(t[n2], invH);
    }
    if (__any_sync(0xffffffffu, big > thrH)) {
      uint32_t mask = 0;
#pragma unroll
      for (int n2 = 0; n2 < S; ++n2) {
        if constexpr (EXT) {
          const float ax = fabsf(t[n2].x), ay = fabsf(t[n2].y);
          const uint32_t lag = (uint32_t)(2 * (n1 + F * n2));
          mask |= (ax > thrH && ax < hiH && lag < a.lag_end ? 1u : 0u) << (2 * n2);
          mask |= (ay > thrH && ay < hiH && lag + 1u < a.lag_end ? 1u : 0u) << (2 * n2 + 1);
        } else {
          mask |= (fabsf(t[n2].x) > thrH ? 1u : 0u) << (2 * n2);
          mask |= (fabsf(t[n2].y) > thrH ? 1u : 0u) << (2 * n2 + 1);
        }
      }
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
      for (int n2 = 0; n2 < S; ++n2) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if ((mask >> (2 * n2 + e)) & 1u) {
            if (pos < a.cap) {
              bege_tail* r = a.recs + pos;
              r->tmpl = tmpl;
              r->lag = (uint32_t)(2 * (n1 + F * n2) + e);
              r->value = (e ? t[n2].y : t[n2].x) * invH;
            }
            ++pos;
            if constexpr (EXT) {
              // positive values above the threshold: v > thr > 0, so the
              // bits of v / sigma order like the values; equal values keep
              // the smaller template (larger ~tmpl)
              const float v = (e ? t[n2].y : t[n2].x) * invH;
              if (a.proj && v > thr)
                atomicMax(a.proj + (2 * (n1 + F * n2) + e),
                          ((unsigned long long)__float_as_uint(v * (1.0f / sigma)) << 32) |
                              (unsigned long long)(~tmpl));
            }
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Interleaved columns (F = 4096, NC = 2, 256 threads, HALFZ templates).
// Row i of the CTA's two columns is the float4 {slot 0 [i], slot 1 [i]} at
// padded row index pad(i) (the same bytes as two separate padded columns).
// In these passes a thread owns butterfly j of both columns, so a pass is
// one round: every load before its barrier, every store after it.  A pass
// can therefore also change the layout, and an interleaved row moves with
// one 16-byte access; a Stockham twiddle (a function of the row, not of the
// column) is loaded once for both columns.  The forward passes end in the
// separate layout, where the fused middle's mirror accesses are free of bank
// conflicts; the inverse passes end interleaved, so the combine reads a
// unit's two columns with one load.  Every value sees the same arithmetic
// in the same order as in the separate layout, and the fused middle keeps
// its thread-to-item map, so the results are bitwise the same.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4* il_rows() { return reinterpret_cast<float4*>(smem_raw); }
__device__ __forceinline__ float4 il_pack(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// The interleaved kernel calls its passes and its fused middle as separate
// (not inlined) functions: each stage then gets the whole register budget
// of the 128-register launch shape to itself, where the inlined kernel
// spilled 100 bytes a thread (two butterflies of data per pass and per
// fused middle).  Measured on 65536 chirps: N = 2^15 6.71 -> 6.66 ms, 2^16
// 14.43 -> 14.16, 2^17 33.1 -> 31.0; at N = 2^14 (no cluster, S = 2) the
// separate layout stays (3.25 against 3.26-3.30 ms).

// Row loads and stores of both columns at padded row index i: interleaved
// (IL, one 16-byte access) or from the two separate columns.
template <bool IL>
__device__ __forceinline__ void il_load(int i, float2& a, float2& b) {
  if constexpr (IL) {
    const float4 v = il_rows()[i];
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
  } else {
    a = Smem<4096, 2>::col(0)[i];
    b = Smem<4096, 2>::col(1)[i];
  }
}
template <bool IL>
__device__ __forceinline__ void il_store(int i, float2 a, float2 b) {
  if constexpr (IL) {
    il_rows()[i] = il_pack(a, b);
  } else {
    Smem<4096, 2>::col(0)[i] = a;
    Smem<4096, 2>::col(1)[i] = b;
  }
}

// First forward pass (radix 16, Ns = 1) of both columns from the template's
// nz <= F/2 complex samples: u_c[m1] = wH^(b_c m1) z[m1], upper half zero.
template <bool OUT_IL>
__device__ __noinline__ void il_fwd_first_pass(const float* __restrict__ src, int nz) {
  using SM = Smem<4096, 2>;
  const float2* z = reinterpret_cast<const float2*>(src);
  const int j = threadIdx.x;
  float2 va[16], vb[16];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int m1 = j + r * 256;
    va[r] = vb[r] = m1 < nz ? __ldg(z + m1) : make_float2(0.f, 0.f);
  }
  const float2 ta = SM::twin()[j], tb = SM::twin()[256 + j];
  const float2* ra = SM::rin();
  const float2* rb = SM::rin() + 16;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    va[r] = cmul(cmul(va[r], ta), ra[r]);
    vb[r] = cmul(cmul(vb[r], tb), rb[r]);
  }
  dft<16, false, true>(va);
  dft<16, false, true>(vb);
  const int q = pad(16 * j);
#pragma unroll
  for (int r = 0; r < 16; ++r) il_store<OUT_IL>(q + r, va[r], vb[r]);
  __syncthreads();
}

// One radix-16 Stockham pass (NB = 256 butterflies per column, Ns = NS) of
// both columns, in one round: every load before the barrier, every store
// after it, so the pass may also change the layout (IN_IL -> OUT_IL).
// Ends with a barrier.
template <int NS, bool INV, bool IN_IL, bool OUT_IL>
__device__ __noinline__ void il_pass(const float2* tw) {
  constexpr int step = 256 + 16;  // padded distance of rows j + 256 r
  static_assert(NS % 16 == 0, "strided stores");
  const int j = threadIdx.x;
  const int k = j & (NS - 1);
  float2 va[16], vb[16];
  const int p = pad(j);
#pragma unroll
  for (int r = 0; r < 16; ++r) il_load<IN_IL>(p + r * step, va[r], vb[r]);
  const float2* t = tw + k;
#pragma unroll
  for (int r = 1; r < 16; ++r) {
    const float2 w = t[r * NS];
    va[r] = INV ? cmulc(va[r], w) : cmul(va[r], w);
    vb[r] = INV ? cmulc(vb[r], w) : cmul(vb[r], w);
  }
  dft<16, INV>(va);
  dft<16, INV>(vb);
  __syncthreads();
  const int q = pad((j - k) * 16 + k);
#pragma unroll
  for (int r = 0; r < 16; ++r) il_store<OUT_IL>(q + r * (NS + NS / 16), va[r], vb[r]);
  __syncthreads();
}

// Last inverse pass (radix 16, Ns = F/16) of both columns with the output
// twiddle T_b[n1] = wH^(-b n1) x[n1] (as inv_last_pass), in one round;
// writes the interleaved layout.  TRAIL: end with a barrier.
template <int S, bool IN_IL, bool TRAIL>
__device__ __noinline__ void il_inv_last_pass() {
  using SM = Smem<4096, 2>;
  constexpr int Ns = 256, step = 256 + 16;
  const int j = threadIdx.x;
  float2 va[16], vb[16];
  const int p = pad(j);
#pragma unroll
  for (int r = 0; r < 16; ++r) il_load<IN_IL>(p + r * step, va[r], vb[r]);
  const float2* t3 = SM::tw3() + j;
#pragma unroll
  for (int r = 1; r < 16; ++r) {
    const float2 w = t3[r * Ns];
    va[r] = cmulc(va[r], w);
    vb[r] = cmulc(vb[r], w);
  }
  dft<16, true>(va);
  dft<16, true>(vb);
  {
    const float2 ta = SM::twin()[j], tb = SM::twin()[256 + j];
    const float2* ra = SM::rout();
    const float2* rb = SM::rout() + 16;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      va[r] = cmul(cmulc(va[r], ta), ra[r]);
      vb[r] = cmul(cmulc(vb[r], tb), rb[r]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) il_store<true>(p + r * step, va[r], vb[r]);
  if constexpr (TRAIL) __syncthreads();
}

// The CTA's share of sum |Y|^2: in its sigpart slot, and with SIGPUSH also
// in slot grank of every CTA's sigall array.
template <int F, int S, int NC, bool SIGPUSH>
__device__ __forceinline__ void store_sigma_partial(int grank, float s) {
  using SM = Smem<F, NC>;
  *SM::sigpart() = s;
  if constexpr (SIGPUSH) {
    constexpr int C = ColMap<S, NC>::C;
    cg::cluster_group cluster = cg::this_cluster();
#pragma unroll
    for (int q = 0; q < C; ++q) *cluster.map_shared_rank(SM::sigall() + grank, (unsigned)q) = s;
  }
}

// S2-S5 for one template on this CTA's columns; leaves the CTA's share of
// sum |Y|^2 in its sigpart slot and T_b in its columns (the caller
// synchronises the cluster before the combine).
//
// SIGPUSH: the CTA's partial is also stored into slot grank of every CTA's
// sigall array, so each CTA sums the cluster's partials from its own memory
// after the next cluster barrier (slot q is rewritten only after the
// barrier that follows every CTA's read of it).
//
// IL: interleaved columns (F = 4096, NC = 2, T = 256, HALFZ, S >= 2 only).
template <int F, int S, int NC, int T, bool HALFZ, bool SIGPUSH = false, bool IL = false>
__device__ __forceinline__ void template_columns(int grank, const float* __restrict__ src, int nz,
                                                 int nfold, const float4* __restrict__ AB,
                                                 int s_rt = S) {
  using SM = Smem<F, NC>;
  constexpr int UPC = S == 1 ? 1 : NC / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if constexpr (IL) {
    static_assert(F == 4096 && NC == 2 && T == 256 && HALFZ && S != 1, "interleaved shape");
    // the forward passes end in the separate layout (the fused middle's
    // mirror accesses are conflict-free there); the inverse passes write
    // the interleaved one, which the combine reads a row at a time
    il_fwd_first_pass<true>(src, nz);
    il_pass<16, false, true, false>(SM::tw2());
    fused_mid_call<S, NC, T>(grank, AB, SM::red());
    if (threadIdx.x == 0) {
      float s = 0.f;
      for (int w = 0; w < T / 32; ++w) s += SM::red()[w];
      store_sigma_partial<F, S, NC, SIGPUSH>(grank, s);
    }
    __syncthreads();
    il_pass<16, true, false, true>(SM::tw2());
    il_inv_last_pass<S, true, !SIGPUSH>();  // without it, a cluster barrier follows
  } else if constexpr (F == 4096) {
    // S2: forward passes 1-2; S2-S5 fused: forward pass 3, the product
    // Y = conj(Z) A + Z' B with sum |Y|^2, inverse pass 1; S5: passes 2-3
    fwd_first_pass<F, S, NC, T, HALFZ>(grank, src, nz, nfold, s_rt);
    stockham_pass<F, NC, T, 16, 16, false>(SM::cols(), SM::tw2());
    fused_mid<S, NC, T>(grank, AB, SM::red(), s_rt);
    if (threadIdx.x == 0) {
      float s = 0.f;
      for (int w = 0; w < T / 32; ++w) s += SM::red()[w];
      store_sigma_partial<F, S, NC, SIGPUSH>(grank, s);
    }
    __syncthreads();
    // rounds of these two passes touch disjoint columns, so (with two or
    // more rounds) a later round's barrier orders the first pass's stores
    // before the second pass's loads
    stockham_pass<F, NC, T, 16, 16, true, false>(SM::cols(), SM::tw2());
    inv_last_pass<F, S, NC, T, !SIGPUSH>();  // without it, a cluster barrier follows
  } else {
    // S2: template spectrum (column FFTs of the packed, twiddled template)
    forward_columns<F, S, NC, T, HALFZ>(grank, src, nz, nfold);
    // S3 + S4: Y = conj(Z) A + Z' B over this CTA's bin pairs, sum |Y|^2
    float acc = 0.f;
#pragma unroll
    for (int ui = 0; ui < UPC; ++ui) {
      const int ug = grank * UPC + ui;
      const int count = unit_items<F, S>(ug);
#pragma unroll 2
      for (int it = threadIdx.x; it < count; it += T) {
        const PairItem q = pair_item<F, S>(ug, ui, it);
        float2* cj = SM::col(q.sj) + pad(q.a);
        float2* cp = SM::col(q.sp) + pad(q.ap);
        const float4 abj = __ldcg(AB + q.b * F + q.a);
        const float4 abp = __ldcg(AB + q.bp * F + q.ap);
        const float2 zj = *cj, zp = *cp;
        const float2 yj = packed_product(zj, zp, abj);
        acc = fmaf(yj.x, yj.x, fmaf(yj.y, yj.y, acc));
        if (cj != cp) {
          const float2 yp = packed_product(zp, zj, abp);
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
      for (int w = 0; w < T / 32; ++w) s += SM::red()[w];
      store_sigma_partial<F, S, NC, SIGPUSH>(grank, s);
    }
    // S5: inverse column FFTs (the first pass reads after the barrier above)
    inverse_columns<F, S, NC, T>();
  }
}

// sigma from the sum |Y|^2 partials of the C CTAs of a group (Eq. PT on the
// packed spectrum: sigma^2 = 2 sum |Y|^2 / N^2).
// The same with the group's CTA count C given at run time.
__device__ __forceinline__ float group_sigma_rt(float* sigpart, int gbase, int C, int N) {
  cg::cluster_group cluster = cg::this_cluster();
  float tot = 0.f;
  for (int q = 0; q < C; ++q) tot += *cluster.map_shared_rank(sigpart, (unsigned)(gbase + q));
  return sqrtf(2.0f * tot) / (float)N;
}

template <int S, int NC>
__device__ __forceinline__ float group_sigma(float* sigpart, int gbase, int N) {
  constexpr int C = ColMap<S, NC>::C;
  cg::cluster_group cluster = cg::this_cluster();
  float tot = 0.f;
#pragma unroll
  for (int q = 0; q < C; ++q)
    tot += *cluster.map_shared_rank(sigpart, (unsigned)(gbase + q));
  return sqrtf(2.0f * tot) / (float)N;
}

// A cluster barrier that orders only earlier reads of distributed shared
// memory before later writes (the combine's remote reads before the next
// template overwrites the columns): every remote value has fed a warp vote
// or the threshold before its thread arrives, so the reads have completed
// and the arrive needs no release fence.  Data that other CTAs read later
// is published by the full (release / acquire) barrier before the combine.
__device__ __forceinline__ void cluster_sync_after_reads() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" :::
               "memory");
}

//
// IL: the CTA's two columns interleaved (F = 4096, NC = 2, T = 256, HALFZ,
// S >= 2); the results are the same bit for bit.
template <int F, int S, int NC, int T, int MINB, bool HALFZ, bool EXT, bool IL = false>
__global__ void __launch_bounds__(T, MINB) correlate_kernel(PlanDev p, CorrelateArgs a) {
  constexpr int C = ColMap<S, NC>::C;
  cg::cluster_group cluster = cg::this_cluster();
  const int N = p.g.N, H = p.g.H;
  const int rank = (int)cluster.block_rank();
  setup_common<F, NC, T>(p);
  setup_columns<F, S, NC, T>(p, rank, 0, !IL);
  if constexpr (IL) {  // the C CTAs' row arrays, for the combine
    if (threadIdx.x < C)
      Smem<F, NC>::colptr()[threadIdx.x] =
          reinterpret_cast<float2*>(cluster.map_shared_rank(il_rows(), (unsigned)threadIdx.x));
  }
  __syncthreads();

  const int cid = blockIdx.x / C;
  const int ncl = gridDim.x / C;
  const int nz = (int)(a.Lp / 2);
  const int nfold = (nz + F - 1) / F;
  const TailOut out{a.recs, a.cap, a.counter, a.dump, a.proj, a.kappa_hi, a.lag_end};

  for (int64_t k = a.k0 + cid; k < a.k1; k += ncl) {
    template_columns<F, S, NC, T, HALFZ, true, IL>(rank, a.bank + k * a.Lp, nz, nfold, a.AB);
    cluster.sync();  // every column and every sigma partial of the cluster is ready
    float sigma;
    {  // Eq. PT over the cluster's partials, summed in rank order as group_sigma does
      float tot = 0.f;
#pragma unroll
      for (int q = 0; q < C; ++q) tot += Smem<F, NC>::sigall()[q];
      sigma = sqrtf(2.0f * tot) / (float)N;
    }
    const int64_t krow = k - a.k0;
    if (rank == 0 && threadIdx.x == 0) a.sigma[krow] = sigma;
    // S6: S-point combine, threshold, warp-ballot compaction
    combine_and_emit<F, S, NC, T, EXT, IL>(Smem<F, NC>::colptr(), H, rank, a.kappa * sigma,
                                           (uint32_t)k, krow, out, sigma);
    cluster_sync_after_reads();  // remote reads done before the columns are overwritten
  }
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
template <typename K>
static cudaError_t ensure_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int F, int S, int NC, int T, int MINB, bool HALFZ, bool EXT>
static cudaError_t launch_corr_tp(const PlanDev& p, const CorrelateArgs& a, cudaStream_t s) {
  constexpr int C = ColMap<S, NC>::C;
  constexpr size_t smem = Lay<F, NC>::total;
  // interleaved columns for S >= 4 (N >= 2^15)
  constexpr bool kIL = (F == 4096 && S >= 4 && NC == 2 && T == 256 && HALFZ);
  auto kern = correlate_kernel<F, S, NC, T, MINB, HALFZ, EXT, kIL>;
  cudaError_t e = ensure_smem(kern, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(T, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  cfg.gridDim = dim3((unsigned)(sms / C * C * MINB), 1, 1);
  int max_clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (max_clusters < 1) return cudaErrorInvalidConfiguration;
  int64_t want = a.k1 - a.k0;
  if (a.max_clusters > 0 && want > a.max_clusters) want = a.max_clusters;
  if (want > max_clusters) want = max_clusters;
  cfg.gridDim = dim3((unsigned)(want * C), 1, 1);
  return cudaLaunchKernelEx(&cfg, kern, p, a);
}

// The extended epilogue (bege_correlate_max, bege_correlate_band,
// bege_correlate_ex) runs in its own instantiation.
template <int F, int S, int NC, int T, int MINB, bool HALFZ>
static cudaError_t launch_corr_t(const PlanDev& p, const CorrelateArgs& a, cudaStream_t s) {
  const bool ext = a.proj || a.kappa_hi > 0.f || a.lag_end < (uint32_t)p.g.N;
  return ext ? launch_corr_tp<F, S, NC, T, MINB, HALFZ, true>(p, a, s)
             : launch_corr_tp<F, S, NC, T, MINB, HALFZ, false>(p, a, s);
}

template <int F, int S, int NC, int T>
static cudaError_t launch_segment_t(const PlanDev& p, const float* y, float2* D, float4* AB,
                                    cudaStream_t s) {
  constexpr size_t smem = Lay<F, NC>::total;
  auto kern = segment_kernel<F, S, NC, T>;
  cudaError_t e = ensure_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<ColMap<S, NC>::C, T, smem, s>>>(p, y, D, AB);
  return cudaGetLastError();
}

}  // namespace bege
