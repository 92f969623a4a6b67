// Device tables of the batching form (shared by bege_batch.cu and the host
// layer).  Not part of the public ABI.
#pragma once

#include "bege_internal.h"

namespace bege {

// One segment of a batch and the bank range it is correlated with.
struct BatchSeg {
  const float4* AB;            // product coefficients of the segment (residue-major)
  const float* bank;           // bank rows of Lp floats
  int64_t Lp;
  int64_t k0, k1;              // bank rows [k0, k1)
  float kappa;
  int S;                       // columns = N / 8192
  float* sigma;                // k1 - k0 floats
  bege_tail* recs;             // tail records of this segment
  uint64_t cap;
  unsigned long long* counter;
};

// A work item: rows [k_begin, k_end) of segment `seg`.
struct BatchItem {
  int seg;
  int pad;
  int64_t k_begin, k_end;
};

// One block of the batched segment-spectrum kernel.
struct SegJob {
  const float* y;
  float2* D;
  float4* AB;
  int S;
  int rank;
};

struct BatchArgs {
  PlanDev plans[4];            // N = 2^14, 2^15, 2^16, 2^17
  const BatchSeg* segs;
  const BatchItem* items;
  int n_items;
  unsigned int* queue;         // next item; zeroed before every launch
};

// Clusters of 8 CTAs of the batch kernel that fit on the device at once.
int batch_max_clusters();
cudaError_t launch_batch(const BatchArgs& b, int clusters, cudaStream_t s);
cudaError_t launch_segment_batch(const BatchArgs& b, const SegJob* jobs, int njobs,
                                 cudaStream_t s);

}  // namespace bege
