// Correlate kernel of the precision form: S2-S6 per template with the column
// FFTs on tcgen05 tensor cores (see bege_tc.cuh for the scheme).
#include "bege_tc.cuh"

namespace bege {
namespace tc {

// GEMM step: operand writes are made visible to the tensor cores, the block
// synchronises, thread 0 issues the MMAs and every thread waits (bounded) on
// the mbarrier.  Returns false if the wait gave up.
template <int P>
__device__ __forceinline__ bool gemm(uint32_t tmem, bool a_mn, int K, uint32_t mbar,
                                     uint32_t& parity) {
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    issue_gemm<P>(tmem, a_mn, K, mbar);
  }
  const bool ok = mbar_wait(mbar, parity);
  parity ^= 1u;
  asm volatile("tcgen05.fence::after_thread_sync;");
  return ok;
}

// Accumulator rows of this thread's warp: rows 32 (warp % 4) + lane,
// complex outputs 32 (warp / 4) + i, i < 32 (columns 2 i, 2 i + 1).
__device__ __forceinline__ void read_rows(uint32_t tmem, float (&v0)[32], float (&v1)[32]) {
  const int w = threadIdx.x >> 5;
  const uint32_t addr = tmem + ((uint32_t)(32 * (w & 3)) << 16) + 64u * (uint32_t)(w >> 2);
  tmem_ld32(addr, v0);
  tmem_ld32(addr + 32, v1);
}

__device__ __forceinline__ float2 outv(const float (&v0)[32], const float (&v1)[32], int i) {
  return i < 16 ? make_float2(v0[2 * i], v0[2 * i + 1]) : make_float2(v1[2 * i - 32], v1[2 * i - 31]);
}

// After the first GEMM of a transform: twiddle w4096^(m1 k1) and write the
// second GEMM's operand MN-major (rows k1, K index m1).
template <int P>
__device__ __forceinline__ void twiddle_to_mn(uint32_t tmem, unsigned char* a_hi,
                                              unsigned char* a_lo) {
  float v0[32], v1[32];
  read_rows(tmem, v0, v1);
  const int w = threadIdx.x >> 5, r = 32 * (w & 3) + (threadIdx.x & 31), h = w >> 2;
  const int c = r >> 6, m1 = r & 63;
#pragma unroll
  for (int blk = 0; blk < 4; ++blk) {
    float re[8], im[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int i = 8 * blk + e, k1 = 32 * h + i;
      const float2 x = cmul(outv(v0, v1, i), w4096<P>(m1 * k1));
      re[e] = x.x;
      im[e] = x.y;
    }
    const int row0 = 64 * c + 32 * h + 8 * blk;
    store_split8<P>(a_hi, a_lo, off_mnmajor(row0, kperm(0, m1)), re);
    store_split8<P>(a_hi, a_lo, off_mnmajor(row0, kperm(1, m1)), im);
  }
}

// Largest |component| over the block (all threads get it); `red` holds 8
// floats of scratch in shared memory.
__device__ __forceinline__ float block_max(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float m = red[0];
#pragma unroll
  for (int w = 1; w < kT / 32; ++w) m = fmaxf(m, red[w]);
  return m;
}

// Power of two s with m s in [256, 512): FP16 operands of the 64-term GEMMs
// then neither overflow nor lose their low parts to subnormals.  Scaling by
// a power of two is exact and is undone after the transform.
__device__ __forceinline__ float pow2_scale(float m) {
  return m > 0.f ? ldexpf(1.0f, 8 - ilogbf(m)) : 1.0f;
}

template <int S, int P>
__global__ void __launch_bounds__(kT, 1) correlate_tc_kernel(PlanDev p, CorrelateArgs a) {
  using SM = Smem<P>;
  using L = TcLay<P>;
  using CM = ColMap<S, kNC>;
  constexpr int C = CM::C;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  const int H = p.g.H, N = p.g.N;
  unsigned char* const a_hi = smem_raw + L::a_hi;
  unsigned char* const a_lo = smem_raw + L::a_lo;
  unsigned char* const b_hi = smem_raw + L::b_hi;
  unsigned char* const b_lo = smem_raw + L::b_lo;
  const uint32_t mbar = smem_addr(smem_raw + L::mbar);
  uint32_t* const tslot = reinterpret_cast<uint32_t*>(smem_raw + L::tslot);

  // ---- set-up: twiddle tables (FP64 -> FP32), DFT matrix parts, column
  // addresses, mbarrier, tensor memory
  const int bcol[2] = {CM::slot_column(rank, 0), CM::slot_column(rank, 1)};
  if (tid < 64) {
    SM::w64()[tid] = root(tid, 64);
    SM::w4k()[tid] = root(tid, 4096);
  }
  for (int i = tid; i < 256; i += kT) {
    const int c = i >> 7, x = i & 63;
    const int64_t b = bcol[c];
    if ((i & 64) == 0)
      SM::tin_a()[c * 64 + x] = root(b * x, H);
    else
      SM::tin_b()[c * 64 + x] = root(64 * b * x, H);
  }
  if (tid < S) {
    int owner, slot;
    CM::home(tid, &owner, &slot);
    SM::colptr()[tid] = cluster.map_shared_rank(SM::col(0), (unsigned)owner) + slot * L::CS;
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();  // w64 ready for the DFT matrix
  // B[n][K]: n = 2 nc + po (output index, re/im), K = kperm(pi, mc) (input)
  for (int i = tid; i < 128 * 128; i += kT) {
    const int n = i >> 7, K = i & 127;
    const int nc = n >> 1, po = n & 1;
    const int mc = ((K >> 6) << 5) | (K & 31), pi = (K >> 5) & 1;
    const float2 wv = SM::w64()[(mc * nc) & 63];
    const float v = po == 0 ? (pi == 0 ? wv.x : -wv.y) : (pi == 0 ? wv.y : wv.x);
    using PT = Part<P>;
    const typename PT::T hv = PT::cvt(v);
    *reinterpret_cast<typename PT::T*>(b_hi + off_kmajor(n, K)) = hv;
    if (P == BF16X3)
      *reinterpret_cast<typename PT::T*>(b_lo + off_kmajor(n, K)) = PT::cvt(v - PT::back(hv));
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;

  const int cid = blockIdx.x / C;
  const int ncl = gridDim.x / C;
  const int nz = (int)(a.Lp / 2);
  const TailOut out{a.recs, a.cap, a.counter, a.dump};
  uint32_t parity = 0;
  bool ok = true;
  const int warp = tid >> 5, lane = tid & 31;

  for (int64_t k = a.k0 + cid; k < a.k1; k += ncl) {
    // ---- forward GEMM 1 operand: u_c[m1 + 64 m2] = wH^(b m) z[m], K-major
    const float2* z = reinterpret_cast<const float2*>(a.bank + k * a.Lp);
    float ure[2][8], uim[2][8];
    float umax = 0.f;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int u = tid + i * kT;
      const int m1 = u & 63, blk = (u >> 6) & 3, c = u >> 8;
      const float2 ta = SM::tin_a()[c * 64 + m1];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int m2 = 8 * blk + e, m = m1 + 64 * m2;
        float2 v = m < nz ? __ldg(z + m) : make_float2(0.f, 0.f);
        v = cmul(cmul(v, ta), SM::tin_b()[c * 64 + m2]);
        ure[i][e] = v.x;
        uim[i][e] = v.y;
        umax = fmaxf(umax, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
    }
    float su = 1.f;  // FP16x2: scale of the forward operand
    if constexpr (P == FP16X2) su = pow2_scale(block_max(umax, SM::red() + 16));
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int u = tid + i * kT;
      const int m1 = u & 63, blk = (u >> 6) & 3, c = u >> 8;
      if constexpr (P == FP16X2) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          ure[i][e] *= su;
          uim[i][e] *= su;
        }
      }
      const int row = 64 * c + m1;
      store_split8<P>(a_hi, a_lo, off_kmajor(row, kperm(0, 8 * blk)), ure[i]);
      store_split8<P>(a_hi, a_lo, off_kmajor(row, kperm(1, 8 * blk)), uim[i]);
    }
    ok &= gemm<P>(tmem, false, 64, mbar, parity);        // inputs m2 < 32 only
    twiddle_to_mn<P>(tmem, a_hi, a_lo);
    ok &= gemm<P>(tmem, true, 128, mbar, parity);
    {  // Z[c][k1 + 64 k2] to the FP32 staging columns
      float v0[32], v1[32];
      read_rows(tmem, v0, v1);
      const int r = 32 * (warp & 3) + lane, h = warp >> 2;
      const int c = r >> 6, k1 = r & 63;
      float2* col = SM::col(c);
      const float inv = 1.0f / su;  // exact: su is a power of two
#pragma unroll
      for (int i = 0; i < 32; ++i) col[pad(k1 + 64 * (32 * h + i))] = cscale(outv(v0, v1, i), inv);
    }
    __syncthreads();

    // ---- S3 + S4 in FP32: Y = conj(Z) A + Z' B over the unit's bin pairs
    float acc = 0.f, ymax = 0.f;
    {
      const int ug = rank;
      const int count = unit_items<kF, S>(ug);
      for (int it = tid; it < count; it += kT) {
        const PairItem q = pair_item<kF, S>(ug, 0, it);
        float2* cj = SM::col(q.sj) + pad(q.a);
        float2* cp = SM::col(q.sp) + pad(q.ap);
        const float4 abj = __ldcg(a.AB + q.b * kF + q.a);
        const float4 abp = __ldcg(a.AB + q.bp * kF + q.ap);
        const float2 zj = *cj, zp = *cp;
        const float2 yj = cadd(cconjmul(zj, make_float2(abj.x, abj.y)),
                               cmul(zp, make_float2(abj.z, abj.w)));
        acc = fmaf(yj.x, yj.x, fmaf(yj.y, yj.y, acc));
        ymax = fmaxf(ymax, fmaxf(fabsf(yj.x), fabsf(yj.y)));
        if (cj != cp) {
          const float2 yp = cadd(cconjmul(zp, make_float2(abp.x, abp.y)),
                                 cmul(zj, make_float2(abp.z, abp.w)));
          acc = fmaf(yp.x, yp.x, fmaf(yp.y, yp.y, acc));
          ymax = fmaxf(ymax, fmaxf(fabsf(yp.x), fabsf(yp.y)));
          *cp = yp;
        }
        *cj = yj;
      }
    }
    float sy = 1.f;  // FP16x2: scale of the inverse operand
    if constexpr (P == FP16X2) sy = pow2_scale(block_max(ymax, SM::red() + 16));
    acc = warp_sum(acc);
    if (lane == 0) SM::red()[warp] = acc;
    __syncthreads();
    if (tid == 0) {
      float s = 0.f;
      for (int w = 0; w < kT / 32; ++w) s += SM::red()[w];
      *SM::sigpart() = s;
    }

    // ---- inverse transform as conj(DFT(conj(Y))): GEMM 1 operand, K-major
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int u = tid + i * kT;
      const int a1 = u & 63, blk = (u >> 6) & 7, c = u >> 9;
      const float2* col = SM::col(c);
      float re[8], im[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float2 y = col[pad(a1 + 64 * (8 * blk + e))];
        re[e] = y.x * sy;
        im[e] = -y.y * sy;
      }
      const int row = 64 * c + a1;
      store_split8<P>(a_hi, a_lo, off_kmajor(row, kperm(0, 8 * blk)), re);
      store_split8<P>(a_hi, a_lo, off_kmajor(row, kperm(1, 8 * blk)), im);
    }
    ok &= gemm<P>(tmem, false, 128, mbar, parity);
    twiddle_to_mn<P>(tmem, a_hi, a_lo);
    ok &= gemm<P>(tmem, true, 128, mbar, parity);
    {  // T_b[n1] = wH^(-b n1) conj(D), n1 = n1a + 64 n1b, to the staging columns
      float v0[32], v1[32];
      read_rows(tmem, v0, v1);
      const int r = 32 * (warp & 3) + lane, h = warp >> 2;
      const int c = r >> 6, n1a = r & 63;
      const float2 ta = SM::tin_a()[c * 64 + n1a];
      float2* col = SM::col(c);
      const float inv = 1.0f / sy;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int n1b = 32 * h + i;
        const float2 x = cscale(cconj(outv(v0, v1, i)), inv);
        col[pad(n1a + 64 * n1b)] = cmulc(cmulc(x, ta), SM::tin_b()[c * 64 + n1b]);
      }
    }

    cluster.sync();  // every column and sigma partial of the cluster is ready
    const float sigma = group_sigma<S, kNC>(SM::sigpart(), 0, N);
    const int64_t krow = k - a.k0;
    if (rank == 0 && tid == 0) a.sigma[krow] = sigma;
    combine_and_emit<kF, S, kNC, kT>(SM::colptr(), H, rank, a.kappa * sigma, (uint32_t)k, krow,
                                     out);
    cluster.sync();  // remote reads done before the staging columns are overwritten
  }

  if (!ok && a.status) atomicOr(a.status, 1u);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                             "r"(kTmemCols));
}

template <int S, int P>
cudaError_t launch_tc_t(const PlanDev& p, const CorrelateArgs& a, cudaStream_t s) {
  constexpr int C = ColMap<S, kNC>::C;
  constexpr size_t smem = TcLay<P>::total;
  auto kern = correlate_tc_kernel<S, P>;
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
  cfg.gridDim = dim3((unsigned)(sms / C * C), 1, 1);
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

}  // namespace tc

cudaError_t launch_correlate_tc(const PlanDev& p, const CorrelateArgs& a, int precision,
                                cudaStream_t s) {
  if (a.k1 <= a.k0) return cudaSuccess;
  const int P = precision == 1 ? tc::BF16X3 : tc::FP16X2;
  switch (p.g.S) {
    case 2: return P ? tc::launch_tc_t<2, tc::BF16X3>(p, a, s) : tc::launch_tc_t<2, tc::FP16X2>(p, a, s);
    case 4: return P ? tc::launch_tc_t<4, tc::BF16X3>(p, a, s) : tc::launch_tc_t<4, tc::FP16X2>(p, a, s);
    case 8: return P ? tc::launch_tc_t<8, tc::BF16X3>(p, a, s) : tc::launch_tc_t<8, tc::FP16X2>(p, a, s);
    case 16: return P ? tc::launch_tc_t<16, tc::BF16X3>(p, a, s) : tc::launch_tc_t<16, tc::FP16X2>(p, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bege
