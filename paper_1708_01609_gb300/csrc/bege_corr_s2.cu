// Correlate kernels for S = 2 columns (N = 2^14).
#include "bege_corr.cuh"

namespace bege {

cudaError_t launch_correlate_s2(const PlanDev& p, const CorrelateArgs& a, CorrConfig c,
                                 bool halfz, cudaStream_t s) {
  if (c.nc == 2 && c.threads == 256)
    return halfz ? launch_corr_t<4096, 2, 2, 256, 2, true>(p, a, s)
                 : launch_corr_t<4096, 2, 2, 256, 2, false>(p, a, s);
  return cudaErrorInvalidValue;
}

}  // namespace bege
