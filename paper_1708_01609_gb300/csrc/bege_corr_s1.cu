// Correlate kernels for S = 1 columns (N = 2^10 .. 2^13).
#include "bege_corr.cuh"

namespace bege {

cudaError_t launch_correlate_s1(const PlanDev& p, const CorrelateArgs& a, CorrConfig c,
                                 bool halfz, cudaStream_t s) {
  if (c.nc != 1 || c.threads != 256) return cudaErrorInvalidValue;
  switch (p.g.F) {
    case 512: return launch_corr_t<512, 1, 1, 256, 2, false>(p, a, s);
    case 1024: return launch_corr_t<1024, 1, 1, 256, 2, false>(p, a, s);
    case 2048: return launch_corr_t<2048, 1, 1, 256, 2, false>(p, a, s);
    case 4096:
      return halfz ? launch_corr_t<4096, 1, 1, 256, 2, true>(p, a, s)
                   : launch_corr_t<4096, 1, 1, 256, 2, false>(p, a, s);
    default: break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace bege
