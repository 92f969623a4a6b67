// Correlate kernel for several segments of one length against the same
// templates.  The paper computes a template's transform once for a block of
// segments (Sec. 3.2 ii-iv); here a CTA runs the forward half of a template
// once, keeps its part of the spectrum (32 values per thread) in an
// L2-resident scratch, and then, for each segment, the product with that
// segment's coefficients, the inverse transform, sigma and the tails, with
// exactly the single-segment kernel's arithmetic.
#include "bege_corr.cuh"

namespace bege {

namespace {

constexpr int kF = 4096;
constexpr int kNC = 2;
constexpr int kT = 256;
constexpr int kMinB = 2;

template <int S>
__global__ void __launch_bounds__(kT, kMinB) correlate_multi_kernel(PlanDev p, MultiArgs a) {
  constexpr int C = ColMap<S, kNC>::C;
  using SM = Smem<kF, kNC>;
  cg::cluster_group cluster = cg::this_cluster();
  const int N = p.g.N, H = p.g.H;
  const int rank = (int)cluster.block_rank();
  setup_common<kF, kNC, kT>(p);
  setup_columns<kF, S, kNC, kT>(p, rank, 0, true);
  __syncthreads();

  const int cid = blockIdx.x / C;
  const int ncl = gridDim.x / C;
  const int nz = (int)(a.Lp / 2);
  float2* const scratch = a.scratch + (size_t)blockIdx.x * 32 * kT;

  for (int64_t k = a.k0 + cid; k < a.k1; k += ncl) {
    // S2: forward passes 1-2 (pass 3 runs inside fused_mid for m = 0)
    fwd_first_pass<kF, S, kNC, kT, true>(rank, a.bank + k * a.Lp, nz, 1);
    stockham_pass<kF, kNC, kT, 16, 16, false>(SM::cols(), SM::tw2());
    const int64_t krow = k - a.k0;
    for (int m = 0; m < a.M; ++m) {
      // S3-S5 for segment m: product, sigma partial, inverse transform
      fused_mid<S, kNC, kT, true>(rank, a.AB[m], SM::red(), S, a.M > 1 ? scratch : nullptr,
                                  m > 0);
      if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < kT / 32; ++w) s += SM::red()[w];
        store_sigma_partial<kF, S, kNC, true>(rank, s);
      }
      __syncthreads();
      // two rounds per pass over disjoint columns: the last inverse pass's
      // round barriers order these stores; a cluster barrier follows it
      stockham_pass<kF, kNC, kT, 16, 16, true, false>(SM::cols(), SM::tw2());
      inv_last_pass<kF, S, kNC, kT, false>();
      cluster.sync();  // every column and sigma partial of the cluster is ready
      float tot = 0.f;  // Eq. PT over the cluster's partials, in rank order
#pragma unroll
      for (int q = 0; q < C; ++q) tot += SM::sigall()[q];
      const float sigma = sqrtf(2.0f * tot) / (float)N;
      if (rank == 0 && threadIdx.x == 0) a.sigma[m][krow] = sigma;
      const TailOut out{a.recs[m], a.cap[m], a.counter[m], nullptr};
      combine_and_emit<kF, S, kNC, kT>(SM::colptr(), H, rank, a.kappa * sigma, (uint32_t)k, krow,
                                       out, sigma);
      cluster_sync_after_reads();  // remote reads done before the columns are overwritten
    }
  }
}

template <int S>
cudaError_t launch_multi_t(const PlanDev& p, const MultiArgs& a, cudaStream_t s) {
  constexpr int C = ColMap<S, kNC>::C;
  constexpr size_t smem = Lay<kF, kNC>::total;
  auto kern = correlate_multi_kernel<S>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(kT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  cfg.gridDim = dim3((unsigned)(sms / C * C * kMinB), 1, 1);
  int max_clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (max_clusters < 1) return cudaErrorInvalidConfiguration;
  int64_t want = a.k1 - a.k0;
  if (want > max_clusters) want = max_clusters;
  // the scratch holds kMinB CTAs per SM: the grid never exceeds that
  if (want * C > (int64_t)sms * kMinB) want = (int64_t)sms * kMinB / C;
  cfg.gridDim = dim3((unsigned)(want * C), 1, 1);
  return cudaLaunchKernelEx(&cfg, kern, p, a);
}

}  // namespace

size_t multi_scratch_bytes(int sms) { return (size_t)sms * kMinB * kT * 32 * sizeof(float2); }

cudaError_t launch_correlate_multi(const PlanDev& p, const MultiArgs& a, cudaStream_t s) {
  if (a.k1 <= a.k0 || a.M < 1) return cudaSuccess;
  if (p.g.F != kF || a.Lp > kF || a.M > kMaxMulti) return cudaErrorInvalidValue;
  switch (p.g.S) {
    case 2: return launch_multi_t<2>(p, a, s);
    case 4: return launch_multi_t<4>(p, a, s);
    case 8: return launch_multi_t<8>(p, a, s);
    case 16: return launch_multi_t<16>(p, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bege
