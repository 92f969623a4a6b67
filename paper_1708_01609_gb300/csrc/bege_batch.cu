// Batching form: many segments of different lengths N (2^14 .. 2^17), each
// against its own range of a bank, in one persistent launch.
//
// Every CTA holds two columns (256 threads, two CTAs per SM) and clusters
// have 8 CTAs.  A segment with S = N / 8192 columns needs C = S/2 CTAs per
// template, so a cluster splits into G = 8/C groups that correlate G
// templates of the same segment side by side.  Clusters take work items
// (segment, template range) from a queue in global memory; all CTAs of a
// cluster take the same item, rebuild the column twiddles for its N and run
// the templates with the same per-template body as the single-segment
// kernel (identical arithmetic, hence identical results).  The queue is a
// counter that the batch zeroes before each launch; clusters leave when it
// passes the last item, so nothing waits on anything else.
#include "bege_batch.h"
#include "bege_corr.cuh"

namespace bege {

namespace {

constexpr int kF = 4096;
constexpr int kNC = 2;
constexpr int kT = 256;
constexpr int kCluster = 8;

__device__ __forceinline__ int plan_index(int S) {
  return S == 2 ? 0 : S == 4 ? 1 : S == 8 ? 2 : 3;
}

// Per-item state lives in shared memory: kept in registers across the
// template loop it would push the 128-register budget of the FFT into spills.
struct ItemState {
  BatchSeg sg;
  int64_t k_begin, k_end;
};

// One work item.  The per-template body takes the column count S = N/8192
// at run time, so a single copy of it serves every segment length; only the
// S-point combine is compiled per S.  (With four per-S copies of the body the
// kernel spills about 1 KB per thread under its 128-register budget.)
__device__ __forceinline__ void run_item(const BatchArgs& b, const ItemState* st, int rank) {
  const int S = st->sg.S;
  const int C = S / kNC;
  const int G = kCluster / C;
  cg::cluster_group cluster = cg::this_cluster();
  const int group = rank / C, grank = rank - group * C, gbase = group * C;
  const PlanDev& p = b.plans[plan_index(S)];
  setup_columns<kF, 0, kNC, kT>(p, grank, gbase, true, S);
  __syncthreads();
  const int64_t iters = (st->k_end - st->k_begin + G - 1) / G;
  for (int64_t i = 0; i < iters; ++i) {
    const int64_t k = st->k_begin + i * G + group;
    const bool active = k < st->k_end;  // uniform over the CTAs of a group
    if (active)
      template_columns<kF, 0, kNC, kT, true>(grank, st->sg.bank + k * st->sg.Lp,
                                             (int)(st->sg.Lp / 2), 1, st->sg.AB, S);
    // a one-CTA group reads only its own columns: a CTA barrier suffices
    if (C == 1) __syncthreads(); else cluster.sync();
    if (active) {
      const float sigma = group_sigma_rt(Smem<kF, kNC>::sigpart(), gbase, C, S * 8192);
      const int64_t krow = k - st->sg.k0;
      if (grank == 0 && threadIdx.x == 0) st->sg.sigma[krow] = sigma;
      const TailOut out{st->sg.recs, st->sg.cap, st->sg.counter, nullptr};
      const float thr = st->sg.kappa * sigma;
      float2* const* cp = Smem<kF, kNC>::colptr();
      switch (S) {
        case 2: combine_and_emit<kF, 2, kNC, kT>(cp, S * 4096, grank, thr, (uint32_t)k, krow, out, 0.f); break;
        case 4: combine_and_emit<kF, 4, kNC, kT>(cp, S * 4096, grank, thr, (uint32_t)k, krow, out, 0.f); break;
        case 8: combine_and_emit<kF, 8, kNC, kT>(cp, S * 4096, grank, thr, (uint32_t)k, krow, out, 0.f); break;
        default: combine_and_emit<kF, 16, kNC, kT>(cp, S * 4096, grank, thr, (uint32_t)k, krow, out, 0.f); break;
      }
    }
    // remote reads done before the columns are overwritten
    if (C == 1) __syncthreads(); else cluster_sync_after_reads();
  }
}

__global__ void __launch_bounds__(kT, 2) batch_kernel(BatchArgs b) {
  __shared__ int item_slot;
  __shared__ ItemState st;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  setup_common<kF, kNC, kT>(b.plans[0]);  // F-only tables: the same for every N
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) item_slot = (int)atomicAdd(b.queue, 1u);
    cluster.sync();
    const int idx = *cluster.map_shared_rank(&item_slot, 0u);
    cluster.sync();  // every CTA has read the index before rank 0 takes the next
    if (idx >= b.n_items) break;
    if (threadIdx.x == 0) {
      const BatchItem item = b.items[idx];
      st.sg = b.segs[item.seg];
      st.k_begin = item.k_begin;
      st.k_end = item.k_end;
    }
    __syncthreads();
    run_item(b, &st, rank);
  }
}

// S1 for every segment of the batch: block i computes rank jobs[i].rank of
// segment jobs[i] (S/2 blocks per segment).
__global__ void __launch_bounds__(kT, 1) segment_batch_kernel(BatchArgs b,
                                                             const SegJob* __restrict__ jobs) {
  const SegJob j = jobs[blockIdx.x];
  switch (j.S) {
    case 2: segment_body<kF, 2, kNC, kT>(b.plans[0], j.rank, j.y, j.D, j.AB); break;
    case 4: segment_body<kF, 4, kNC, kT>(b.plans[1], j.rank, j.y, j.D, j.AB); break;
    case 8: segment_body<kF, 8, kNC, kT>(b.plans[2], j.rank, j.y, j.D, j.AB); break;
    default: segment_body<kF, 16, kNC, kT>(b.plans[3], j.rank, j.y, j.D, j.AB); break;
  }
}

}  // namespace

int batch_max_clusters() {
  static int cached = -1;
  if (cached >= 0) return cached;
  constexpr size_t smem = Lay<kF, kNC>::total;
  if (cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(kT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cfg.gridDim = dim3((unsigned)(sms * 2 / kCluster * kCluster), 1, 1);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, batch_kernel, &cfg) != cudaSuccess) n = 0;
  cached = n;
  return n;
}

cudaError_t launch_batch(const BatchArgs& b, int clusters, cudaStream_t s) {
  constexpr size_t smem = Lay<kF, kNC>::total;
  cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(kT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.gridDim = dim3((unsigned)(clusters * kCluster), 1, 1);
  return cudaLaunchKernelEx(&cfg, batch_kernel, b);
}

cudaError_t launch_segment_batch(const BatchArgs& b, const SegJob* jobs, int njobs,
                                 cudaStream_t s) {
  constexpr size_t smem = Lay<kF, kNC>::total;
  cudaError_t e = cudaFuncSetAttribute(segment_batch_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (njobs <= 0) return cudaSuccess;
  segment_batch_kernel<<<njobs, kT, smem, s>>>(b, jobs);
  return cudaGetLastError();
}

}  // namespace bege
