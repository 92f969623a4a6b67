// Geometry, launch-shape tables, the segment-spectrum kernel launcher and
// chirp-bank synthesis.
#include "bege_corr.cuh"

namespace bege {

Geometry make_geometry(int64_t n) {
  Geometry g{};
  g.N = (int)n;
  g.H = g.N / 2;
  g.F = g.H < 4096 ? g.H : 4096;
  g.S = g.H / g.F;
  g.R0 = g.F / 256;
  return g;
}

int correlate_configs(const Geometry& g, CorrConfig* out, int max) {
  CorrConfig all[4];
  int n = 0;
  if (g.S == 1) {
    all[n++] = {1, 256};
  } else if (g.S == 2) {
    all[n++] = {2, 256};
  } else {
    all[n++] = {2, 256};
    all[n++] = {4, 512};
  }
  for (int i = 0; i < n && i < max; ++i) out[i] = all[i];
  return n;
}

bool config_valid(const Geometry& g, CorrConfig c) {
  CorrConfig all[4];
  const int n = correlate_configs(g, all, 4);
  for (int i = 0; i < n; ++i)
    if (all[i].nc == c.nc && all[i].threads == c.threads) return true;
  return false;
}

// Default launch shape: two columns and 256 threads per CTA (two CTAs per
// SM) was the fastest for every N >= 2^14 on GB300.
CorrConfig default_config(const Geometry& g) {
  if (g.S == 1) return {1, 256};
  return {2, 256};
}

cudaError_t launch_segment(const PlanDev& p, const float* y, float2* D, float4* AB,
                           cudaStream_t s) {
  const Geometry& g = p.g;
  switch (g.S) {
    case 1:
      switch (g.F) {
        case 512: return launch_segment_t<512, 1, 1, 256>(p, y, D, AB, s);
        case 1024: return launch_segment_t<1024, 1, 1, 256>(p, y, D, AB, s);
        case 2048: return launch_segment_t<2048, 1, 1, 256>(p, y, D, AB, s);
        case 4096: return launch_segment_t<4096, 1, 1, 256>(p, y, D, AB, s);
        default: return cudaErrorInvalidValue;
      }
    case 2: return launch_segment_t<4096, 2, 2, 256>(p, y, D, AB, s);
    case 4: return launch_segment_t<4096, 4, 4, 512>(p, y, D, AB, s);
    case 8: return launch_segment_t<4096, 8, 4, 512>(p, y, D, AB, s);
    case 16: return launch_segment_t<4096, 16, 4, 512>(p, y, D, AB, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_correlate(const PlanDev& p, const CorrelateArgs& a, CorrConfig cfg,
                             cudaStream_t s) {
  if (a.k1 <= a.k0) return cudaSuccess;
  const Geometry& g = p.g;
  if (!config_valid(g, cfg)) return cudaErrorInvalidValue;
  const bool halfz = (g.F == 4096) && (a.Lp <= g.F);
  switch (g.S) {
    case 1: return launch_correlate_s1(p, a, cfg, halfz, s);
    case 2: return launch_correlate_s2(p, a, cfg, halfz, s);
    case 4: return launch_correlate_s4(p, a, cfg, halfz, s);
    case 8: return launch_correlate_s8(p, a, cfg, halfz, s);
    case 16: return launch_correlate_s16(p, a, cfg, halfz, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// Bank synthesis: w[m] = T(m) sin(2 pi phase(m)), unit L2 norm; time-
// symmetric banks (Fig. 2 caption): w[m] = T(m) (sin(2 pi phase(m)) +
// sin(2 pi phase(L - 1 - m))), the chirp forward and backward in time.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double chirp_sin(unsigned long long alpha, unsigned long long beta,
                                            int64_t m) {
  const unsigned long long um = (unsigned long long)m;
  // phase in cycles * 2^64, exact modulo one cycle
  const unsigned long long ph = alpha * um + beta * (um * um);
  const double c = (double)(long long)ph * 0x1p-64;  // in [-1/2, 1/2)
  return sinpi(2.0 * c);
}

__device__ __forceinline__ double chirp_sample(unsigned long long alpha, unsigned long long beta,
                                               int64_t m, int64_t L, int width, double denom,
                                               bool symmetric) {
  double s = chirp_sin(alpha, beta, m);
  if (symmetric) s += chirp_sin(alpha, beta, L - 1 - m);
  const int64_t mm = m < L - 1 - m ? m : L - 1 - m;
  double t = 1.0;
  if (mm <= width) t = 0.5 * (1.0 - cospi(2.0 * (double)mm / denom));
  return t * s;
}

__global__ void __launch_bounds__(256) bank_chirp_kernel(const unsigned long long* __restrict__ ab,
                                                         int64_t L, int64_t Lp, double frac,
                                                         bool symmetric,
                                                         float* __restrict__ bank) {
  __shared__ double red[8];
  const int64_t k = blockIdx.x;
  const unsigned long long alpha = ab[2 * k], beta = ab[2 * k + 1];
  const int width = (frac > 0.0 && L >= 2) ? (int)floor(frac * (double)(L - 1) / 2.0) : -1;
  const double denom = frac * (double)(L - 1);
  double acc = 0.0;
  for (int64_t m = threadIdx.x; m < L; m += blockDim.x) {
    const double v = chirp_sample(alpha, beta, m, L, width, denom, symmetric);
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
    row[m] = m < L ? (float)(chirp_sample(alpha, beta, m, L, width, denom, symmetric) * scale)
                   : 0.f;
}

cudaError_t launch_bank_chirp(const unsigned long long* alpha_beta, int64_t count, int64_t L,
                              int64_t Lp, double taper_frac, bool symmetric, float* bank,
                              cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  bank_chirp_kernel<<<(unsigned)count, 256, 0, s>>>(alpha_beta, L, Lp, taper_frac, symmetric,
                                                    bank);
  return cudaGetLastError();
}

}  // namespace bege
