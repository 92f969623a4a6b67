// Internal interface between the C-ABI host layer (bege_api.cpp) and the
// CUDA kernels (bege_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bege.h"

namespace bege {

// Geometry of the length-N correlation (N = 2H real samples).
//
// The real N-point transforms are carried by H-point complex transforms of
// the even/odd packed sequence z[m] = x[2m] + i x[2m+1].  The H-point
// transform is split by residue: bin j = S a + b (a < F, b < S) lives in
// "column" b, an F-point FFT of a twiddled, folded input (a four-step whose
// first step is pruned by the template's support).  Columns b and S-b hold
// the bins j and H-j that the real-FFT unpacking couples, so they form a
// "unit" processed by one CTA; the C CTAs of a thread-block cluster share
// the S columns and exchange them through distributed shared memory only for
// the final S-point combine.
struct Geometry {
  int N;    // real samples
  int H;    // N / 2 complex samples
  int F;    // column FFT length (512..4096)
  int S;    // columns = H / F (1..16)
  int R0;   // radix of the first Stockham pass = F / 256
  int C;    // CTAs per cluster
  int NC;   // columns per CTA
  int UPC;  // units per CTA
};

// Device twiddle tables for one N (computed in FP64 on the host, rounded to
// FP32 once).  wX^k means exp(-2 pi i k / X).
struct PlanDev {
  Geometry g;
  const float2* tw2;   // [16*R0]  Stockham pass 2: [r*R0 + k] = w(16 R0)^(k r)
  const float2* tw3;   // [F]      Stockham pass 3: [r*(F/16) + k] = wF^(k r)
  const float2* wH;    // [256*S]  wH^k
  const float2* wR0S;  // [R0*S]   w(R0 S)^q
  const float2* w16S;  // [16*S]   w(16 S)^q
  const float2* wS;    // [S]      wS^q
  const float2* wN;    // [H]      wN^j
};

Geometry make_geometry(int64_t n);

// Shared-memory bytes of the correlate / segment kernels for geometry g.
size_t correlate_smem_bytes(const Geometry& g);

// S1: segment spectrum.  y: N floats (device).  D: H+1 complex (natural
// order).  AB: S*F float4 {A_j, B_j} in residue-major order [b*F + a].
cudaError_t launch_segment(const PlanDev& p, const float* y, float2* D, float4* AB,
                           cudaStream_t s);

// S2..S6 over bank rows [k0, k1).  bank: rows of Lp floats (zero-padded
// beyond L, Lp a multiple of 8).  sigma: k1-k0 floats.  recs/cap/counter:
// tail records.  dump: optional (k1-k0) x N floats of rho.
struct CorrelateArgs {
  const float4* AB;
  const float* bank;
  int64_t Lp;
  int64_t k0, k1;
  float kappa;
  float* sigma;
  bege_tail* recs;
  uint64_t cap;
  unsigned long long* counter;
  float* dump;
  int max_clusters;  // 0 = as many as fit
};
cudaError_t launch_correlate(const PlanDev& p, const CorrelateArgs& a, cudaStream_t s);

// Bank synthesis: count chirps, phase coefficients alpha/beta as unsigned
// 64-bit fixed point (cycles * 2^64), L samples, taper fraction; rows of Lp.
cudaError_t launch_bank_chirp(const unsigned long long* alpha_beta, int64_t count, int64_t L,
                              int64_t Lp, double taper_frac, float* bank, cudaStream_t s);

}  // namespace bege
