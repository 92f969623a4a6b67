// Internal interface between the C-ABI host layer (bege_api.cpp) and the
// CUDA kernels (bege_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

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
// "unit" processed by one CTA; the CTAs of a thread-block cluster share the
// S columns and exchange them through distributed shared memory only for
// the final S-point combine.
struct Geometry {
  int N;    // real samples
  int H;    // N / 2 complex samples
  int F;    // column FFT length (512..4096)
  int S;    // columns = H / F (1..16)
  int R0;   // radix of the first Stockham pass = F / 256
};

// Launch shape of the correlate kernel: columns per CTA (the cluster has
// S / nc CTAs) and threads per CTA.  Chosen per N by default or by the
// autotuner.
struct CorrConfig {
  int nc;
  int threads;
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

// Record `msg` as the calling thread's last error (bege_last_error) and
// return `code`.
int set_last_error(int code, const std::string& msg);

// CUDA device of a context, and the row count of one of its banks (0 if the
// handle is unknown).
int ctx_device(const bege_ctx* ctx);
int64_t bank_count(bege_ctx* ctx, int32_t bank_id);

// Stop every serving-form server of a context.
void serve_destroy_all(bege_ctx* ctx);

// Launch shapes compiled for geometry g (at most `max`); returns the count.
int correlate_configs(const Geometry& g, CorrConfig* out, int max);
CorrConfig default_config(const Geometry& g);
bool config_valid(const Geometry& g, CorrConfig c);

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
  int max_clusters;      // 0 = as many as fit
  unsigned int* status;  // optional: set non-zero by a kernel whose bounded wait gave up
  unsigned long long* proj = nullptr;  // optional: per-lag maximum over the bank (Eq. Ak)
  float kappa_hi = 0.f;                // optional: tails only below kappa_hi sigma (0 = none)
  uint32_t lag_end = 0xffffffffu;      // optional: tails only at lags < lag_end (overlap-save)
};
cudaError_t launch_correlate(const PlanDev& p, const CorrelateArgs& a, CorrConfig cfg,
                             cudaStream_t s);

// Several segments of one length against the same templates (Sec. 3.2: a
// template's transform serves a block of segments): per template the
// forward transform runs once, then the product, inverse, sigma and tails
// for each segment m < M into its own outputs.  F = 4096 (N >= 2^14) and
// Lp <= 4096 only.
constexpr int kMaxMulti = 8;
struct MultiArgs {
  const float* bank;
  int64_t Lp;
  int64_t k0, k1;
  float kappa;
  int M;
  const float4* AB[kMaxMulti];
  float* sigma[kMaxMulti];
  bege_tail* recs[kMaxMulti];
  uint64_t cap[kMaxMulti];
  unsigned long long* counter[kMaxMulti];
  float2* scratch;  // multi_scratch_bytes(): the template spectrum of each CTA
};
size_t multi_scratch_bytes(int sms);
cudaError_t launch_correlate_multi(const PlanDev& p, const MultiArgs& a, cudaStream_t s);

// Per-S launchers (one translation unit each); halfz: Lp <= F.
cudaError_t launch_correlate_s1(const PlanDev& p, const CorrelateArgs& a, CorrConfig c, bool halfz,
                                cudaStream_t s);
cudaError_t launch_correlate_s2(const PlanDev& p, const CorrelateArgs& a, CorrConfig c, bool halfz,
                                cudaStream_t s);
cudaError_t launch_correlate_s4(const PlanDev& p, const CorrelateArgs& a, CorrConfig c, bool halfz,
                                cudaStream_t s);
cudaError_t launch_correlate_s8(const PlanDev& p, const CorrelateArgs& a, CorrConfig c, bool halfz,
                                cudaStream_t s);
cudaError_t launch_correlate_s16(const PlanDev& p, const CorrelateArgs& a, CorrConfig c, bool halfz,
                                 cudaStream_t s);

// Precision form: S2-S6 with the column FFTs on tcgen05 tensor cores.
// precision 1 = BF16x3, 2 = FP16x3.  Needs F = 4096 (N >= 2^14) and
// Lp <= 4096.
cudaError_t launch_correlate_tc(const PlanDev& p, const CorrelateArgs& a, int precision,
                                cudaStream_t s);

// Bank synthesis: count chirps, phase coefficients alpha/beta as unsigned
// 64-bit fixed point (cycles * 2^64), L samples, taper fraction; rows of Lp;
// symmetric: the chirp plus its time reversal (Fig. 2 caption).
cudaError_t launch_bank_chirp(const unsigned long long* alpha_beta, int64_t count, int64_t L,
                              int64_t Lp, double taper_frac, bool symmetric, float* bank,
                              cudaStream_t s);

}  // namespace bege
