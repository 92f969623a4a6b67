// Correlate kernels for S = 4 columns (N = 2^15).
#include "bege_corr.cuh"

namespace bege {

cudaError_t launch_correlate_s4(const PlanDev& p, const CorrelateArgs& a, CorrConfig c,
                                 bool halfz, cudaStream_t s) {
  if (c.nc == 2 && c.threads == 256)
    return halfz ? launch_corr_t<4096, 4, 2, 256, 2, true>(p, a, s)
                 : launch_corr_t<4096, 4, 2, 256, 2, false>(p, a, s);
  if (c.nc == 4 && c.threads == 512)
    return halfz ? launch_corr_t<4096, 4, 4, 512, 1, true>(p, a, s)
                 : launch_corr_t<4096, 4, 4, 512, 1, false>(p, a, s);
  return cudaErrorInvalidValue;
}

}  // namespace bege
