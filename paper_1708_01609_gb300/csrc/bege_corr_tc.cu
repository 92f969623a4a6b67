// Correlate kernel of the precision form: S2-S6 per template with the column
// FFTs on tcgen05 tensor cores (see bege_tc.cuh for the scheme).
#include "bege_tc.cuh"

namespace bege {
namespace tc {

// Barrier of one group's 256 threads (named barrier 1 + g).
__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kGT) : "memory");
}

// GEMM step of group g: operand writes are made visible to the tensor cores,
// the group synchronises, its first thread issues the MMAs and every thread
// waits (bounded) on the group's mbarrier.
//
// Give-up path: a thread whose wait gives up clears `ok` and keeps `parity`
// at the phase it gave up on.  From then on it waits no more, and if it is
// the issuing thread it issues no more MMAs, so the commit of that phase is
// the only one that can still be pending (every earlier phase was waited
// for).  The kernel keeps its barriers in step with the cluster, finishes its
// loop with meaningless values, reports the failure in the job's status word
// and, before releasing tensor memory, the issuing thread waits once more for
// the phase it gave up on (drain_after_give_up).
template <int P>
__device__ __forceinline__ void gemm(int g, int lt, uint32_t tmem, uint32_t ah, uint32_t al,
                                     uint32_t bh, uint32_t bl, bool a_mn, int K, uint32_t mbar,
                                     uint32_t& parity, bool& ok) {
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  group_sync(g);
  if (lt == 0 && ok) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    issue_gemm<P>(tmem, ah, al, bh, bl, a_mn, K, mbar);
  }
  if (ok) {
    if (mbar_wait(mbar, parity))
      parity ^= 1u;
    else
      ok = false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
}

// Before tensor memory is released: if the issuing thread gave up on a
// phase, its commit may still be pending; wait for it once more (bounded).
// Whatever the outcome the failure is already in the job's status word.
__device__ __forceinline__ void drain_after_give_up(int lt, bool ok, uint32_t mbar,
                                                    uint32_t parity) {
  if (lt == 0 && !ok) (void)mbar_wait(mbar, parity);
}

// Half the accumulator row of this thread, in two chunks q = 0, 1: warp w of
// the group reads TMEM lanes 32 (w % 4) + lane, FP32 columns 64 ((w / 4) % 2)
// + 32 q .. + 31 of the group's accumulator, i.e. complex outputs
// 32 ((w / 4) % 2) + 16 q + i, i < 16, as (re, im) in v[2 i], v[2 i + 1].
__device__ __forceinline__ void read_chunk(uint32_t tmem, int q, float (&v)[32]) {
  const int w = threadIdx.x >> 5;
  tmem_ld32(tmem + ((uint32_t)(32 * (w & 3)) << 16) + 64u * (uint32_t)((w >> 2) & 1) +
                32u * (uint32_t)q,
            v);
}

// After the first GEMM of a transform: twiddle w4096^(m1 k1) and write the
// second GEMM's operand MN-major (rows k1, K index m1).  The twiddles of a run
// of 8 outputs come from one table value and the step w4096^m1.
template <int P, int G>
__device__ __forceinline__ void twiddle_to_mn(uint32_t tmem, unsigned char* a_hi,
                                              unsigned char* a_lo) {
  const int w = threadIdx.x >> 5, r = 32 * (w & 3) + (threadIdx.x & 31), h = (w >> 2) & 1;
  const int c = r >> 6, m1 = r & 63;
  const float2 step = w4096<P, G>(m1);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    float v[32];
    read_chunk(tmem, q, v);
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
      const int k0 = 32 * h + 16 * q + 8 * blk;
      float2 tw = w4096<P, G>(m1 * k0);
      float re[8], im[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float2 x = cmul(make_float2(v[16 * blk + 2 * e], v[16 * blk + 2 * e + 1]), tw);
        re[e] = x.x;
        im[e] = x.y;
        tw = cmul(tw, step);
      }
      const int row0 = 64 * c + k0;
      store_split8<P>(a_hi, a_lo, off_mnmajor(row0, kperm(0, m1)), re);
      store_split8<P>(a_hi, a_lo, off_mnmajor(row0, kperm(1, m1)), im);
    }
  }
}

// Largest |component| over group g (all its threads get it); `red` holds 8
// floats of scratch in shared memory.
__device__ __forceinline__ float group_max(int g, float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[(threadIdx.x >> 5) & 7] = v;
  group_sync(g);
  float m = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
  return m;
}

// Power of two s with m s in [256, 512): FP16 operands of the 64-term GEMMs
// then neither overflow nor lose their low parts to subnormals.  Scaling by
// a power of two is exact and is undone after the transform.
__device__ __forceinline__ float pow2_scale(float m) {
  return m > 0.f ? ldexpf(1.0f, 8 - ilogbf(m)) : 1.0f;
}

// G groups of 8 warps per CTA, group g = the CTA's unit g (column slots 2g,
// 2g + 1); clusters of S / (2 G) CTAs hold the S columns of a template.  For
// S = 2 a template is one unit: the two groups of a CTA then take different
// templates (k0 + 2c + g, ...) and never wait for each other.
template <int S, int P, int G>
__global__ void __launch_bounds__(kGT * G, 1) correlate_tc_kernel(PlanDev p, CorrelateArgs a) {
  constexpr bool kInd = (S == 2 && G == 2);  // independent groups
  constexpr int NC = kInd ? 2 : 2 * G;       // columns per CTA in the column map
  constexpr int T = kGT * G;
  using SM = Smem<P, G>;
  using L = TcLay<P, G>;
  using CM = ColMap<S, NC>;
  constexpr int C = CM::C;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  const int g = tid >> 8, lt = tid & (kGT - 1);  // group, thread within the group
  const int H = p.g.H, N = p.g.N;
  unsigned char* const a_hi = smem_raw + L::a_hi(g);
  unsigned char* const a_lo = smem_raw + L::a_lo(g);
  const uint32_t sbase = smem_addr(smem_raw);
  const uint32_t ah = sbase + (uint32_t)L::a_hi(g), al = sbase + (uint32_t)L::a_lo(g);
  const uint32_t bh = sbase + (uint32_t)L::b_hi, bl = sbase + (uint32_t)L::b_lo;
  const uint32_t mbar = sbase + (uint32_t)(L::mbar + 8 * g);
  uint32_t* const tslot = reinterpret_cast<uint32_t*>(smem_raw + L::tslot);
  float* const red = SM::red(g);

  // ---- set-up: twiddle tables (FP64 -> FP32), DFT matrix parts, column
  // addresses, mbarriers, tensor memory
  if (tid < 64) {
    SM::w64()[tid] = root(tid, 64);
    SM::w4k()[tid] = root(tid, 4096);
  }
  for (int i = tid; i < NC * 128; i += T) {
    const int c = i >> 7, x = i & 63;
    const int64_t b = CM::slot_column(rank, c);
    if ((i & 64) == 0)
      SM::tin_a()[c * 64 + x] = root(b * x, H);
    else
      SM::tin_b()[c * 64 + x] = root(64 * b * x, H);
  }
  if constexpr (kInd) {
    if (tid < 2 * S) {  // group gg's columns, in its own region
      const int gg = tid / S, b = tid % S;
      int owner, slot;
      CM::home(b, &owner, &slot);
      SM::colptr()[S * gg + b] = SM::col(2 * gg + slot);
    }
  } else if (tid < S) {
    int owner, slot;
    CM::home(tid, &owner, &slot);
    SM::colptr()[tid] = cluster.map_shared_rank(SM::col(0), (unsigned)owner) + slot * L::CS;
  }
  if (tid < G) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbase + (uint32_t)(L::mbar + 8 * tid)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tslot)),
                 "r"(128u * G));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();  // w64 ready for the DFT matrix
  // B[n][K]: n = 2 nc + po (output index, re/im), K = kperm(pi, mc) (input)
  for (int i = tid; i < 128 * 128; i += T) {
    const int n = i >> 7, K = i & 127;
    const int nc = n >> 1, po = n & 1;
    const int mc = ((K >> 6) << 5) | (K & 31), pi = (K >> 5) & 1;
    const float2 wv = SM::w64()[(mc * nc) & 63];
    const float v = po == 0 ? (pi == 0 ? wv.x : -wv.y) : (pi == 0 ? wv.y : wv.x);
    using PT = Part<P>;
    const typename PT::T hv = PT::cvt(v);
    *reinterpret_cast<typename PT::T*>(smem_raw + L::b_hi + off_kmajor(n, K)) = hv;
    *reinterpret_cast<typename PT::T*>(smem_raw + L::b_lo + off_kmajor(n, K)) =
        PT::cvt(v - PT::back(hv));
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot + 128u * (uint32_t)g;  // the group's accumulator columns

  const int cid = blockIdx.x / C;
  const int ncl = gridDim.x / C;
  const int nz = (int)(a.Lp / 2);
  const TailOut out{a.recs, a.cap, a.counter, a.dump, a.proj, a.kappa_hi, a.lag_end};
  uint32_t parity = 0;
  bool ok = true;
  const int warp = tid >> 5, lane = tid & 31;
  // this thread's accumulator row (TMEM lane), half of the outputs, slot
  const int trow = 32 * (warp & 3) + lane, th = (warp >> 2) & 1;
  const int tslot_ = 2 * g + (trow >> 6), tr = trow & 63;
  const int ttab = kInd ? (trow >> 6) : tslot_;  // its column's twiddle-table slot
  const int ug = kInd ? 0 : rank * CM::UPC + g;  // the group's unit
  const int64_t kfirst = kInd ? a.k0 + 2 * cid + g : a.k0 + cid;
  const int kstride = kInd ? 2 * ncl : ncl;

  for (int64_t k = kfirst; k < a.k1; k += kstride) {
    // ---- forward GEMM 1 operand: u_c[m1 + 64 m2] = wH^(b m) z[m], K-major;
    // the twiddles of a run of 8 m2 from one product and the step wH^(64 b)
    const float2* z = reinterpret_cast<const float2*>(a.bank + k * a.Lp);
    if (k + ncl < a.k1 && tid * 32 < a.Lp)  // the next template's samples to L2
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a.bank + (k + ncl) * a.Lp + tid * 32));
    float ure[2][8], uim[2][8];
    float umax = 0.f;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int u = lt + i * kGT;
      const int m1 = u & 63, blk = (u >> 6) & 3, sl = kInd ? (u >> 8) : 2 * g + (u >> 8);
      float2 zv[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int m = m1 + 64 * (8 * blk + e);
        zv[e] = m < nz ? __ldg(z + m) : make_float2(0.f, 0.f);
      }
      float2 tw = cmul(SM::tin_a()[sl * 64 + m1], SM::tin_b()[sl * 64 + 8 * blk]);
      const float2 step = SM::tin_b()[sl * 64 + 1];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float2 v = cmul(zv[e], tw);
        tw = cmul(tw, step);
        ure[i][e] = v.x;
        uim[i][e] = v.y;
        umax = fmaxf(umax, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
    }
    float su = 1.f;  // FP16x3: scale of the forward operand
    if constexpr (P == FP16X3) su = pow2_scale(group_max(g, umax, red + 16));
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int u = lt + i * kGT;
      const int m1 = u & 63, blk = (u >> 6) & 3, c = u >> 8;
      if constexpr (P == FP16X3) {
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
    gemm<P>(g, lt, tmem, ah, al, bh, bl, false, 64, mbar, parity, ok);  // m2 < 32 only
    twiddle_to_mn<P, G>(tmem, a_hi, a_lo);
    gemm<P>(g, lt, tmem, ah, al, bh, bl, true, 128, mbar, parity, ok);
    {  // Z[c][k1 + 64 k2] to the FP32 staging columns (the A operand is dead)
      float2* col = SM::col(tslot_);
      const float inv = 1.0f / su;  // exact: su is a power of two
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float v[32];
        read_chunk(tmem, q, v);
#pragma unroll
        for (int i = 0; i < 16; ++i)
          col[pad(tr + 64 * (32 * th + 16 * q + i))] =
              make_float2(v[2 * i] * inv, v[2 * i + 1] * inv);
      }
    }
    group_sync(g);

    // ---- S3 + S4 in FP32: Y = conj(Z) A + Z' B over the unit's bin pairs,
    // in place; four items' loads are issued before their arithmetic
    float acc = 0.f, ymax = 0.f;
    if (ug != 0) {
      // unit {b, S-b}: pairs (a, F-1-a) of slots 2g, 2g+1, all distinct
      const int b = ug, bp = S - ug;
      float2* c0 = SM::col(2 * g);
      float2* c1 = SM::col(2 * g + 1);
#pragma unroll 1
      for (int it0 = 0; it0 < kF; it0 += 4 * kGT) {
        float2 zj[4], zp[4];
        float4 abj[4], abp[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int it = it0 + u * kGT + lt, ip = kF - 1 - it;
          abj[u] = __ldcg(a.AB + b * kF + it);
          abp[u] = __ldcg(a.AB + bp * kF + ip);
          zj[u] = c0[pad(it)];
          zp[u] = c1[pad(ip)];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int it = it0 + u * kGT + lt, ip = kF - 1 - it;
          const float2 yj = packed_product(zj[u], zp[u], abj[u]);
          const float2 yp = packed_product(zp[u], zj[u], abp[u]);
          acc = fmaf(yj.x, yj.x, fmaf(yj.y, yj.y, acc));
          acc = fmaf(yp.x, yp.x, fmaf(yp.y, yp.y, acc));
          ymax = fmaxf(ymax, fmaxf(fmaxf(fabsf(yj.x), fabsf(yj.y)), fmaxf(fabsf(yp.x), fabsf(yp.y))));
          c0[pad(it)] = yj;
          c1[pad(ip)] = yp;
        }
      }
    } else {
      // unit {0, S/2}: each column pairs with itself
      const int count = unit_items<kF, S>(ug);
      for (int it0 = 0; it0 < count; it0 += 4 * kGT) {
        float2 zj[4], zp[4];
        float4 abj[4], abp[4];
        int oj[4], op[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int it = it0 + u * kGT + lt;
          oj[u] = -1;
          if (it < count) {
            const PairItem q = pair_item<kF, S>(ug, g, it);
            oj[u] = q.sj * L::CS + pad(q.a);
            op[u] = q.sp * L::CS + pad(q.ap);
            abj[u] = __ldcg(a.AB + q.b * kF + q.a);
            abp[u] = __ldcg(a.AB + q.bp * kF + q.ap);
            zj[u] = SM::col(0)[oj[u]];
            zp[u] = SM::col(0)[op[u]];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (oj[u] < 0) continue;
          const float2 yj = packed_product(zj[u], zp[u], abj[u]);
          acc = fmaf(yj.x, yj.x, fmaf(yj.y, yj.y, acc));
          ymax = fmaxf(ymax, fmaxf(fabsf(yj.x), fabsf(yj.y)));
          if (oj[u] != op[u]) {
            const float2 yp = packed_product(zp[u], zj[u], abp[u]);
            acc = fmaf(yp.x, yp.x, fmaf(yp.y, yp.y, acc));
            ymax = fmaxf(ymax, fmaxf(fabsf(yp.x), fabsf(yp.y)));
            SM::col(0)[op[u]] = yp;
          }
          SM::col(0)[oj[u]] = yj;
        }
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) red[warp & 7] = acc;
    float sy = 1.f;  // FP16x3: scale of the inverse operand
    if constexpr (P == FP16X3)
      sy = pow2_scale(group_max(g, ymax, red + 16));
    else
      group_sync(g);
    if (lt == 0) {
      float s = 0.f;
      for (int w = 0; w < 8; ++w) s += red[w];
      SM::sigpart()[g] = s;
    }

    // ---- inverse transform as conj(DFT(conj(Y))): GEMM 1 operand, K-major.
    // Every Y is read into registers before the operand overwrites the columns.
    {
      float yre[4][8], yim[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int u = lt + i * kGT;
        const int a1 = u & 63, blk = (u >> 6) & 7;
        const float2* col = SM::col(2 * g + (u >> 9));
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float2 y = col[pad(a1 + 64 * (8 * blk + e))];
          yre[i][e] = y.x * sy;
          yim[i][e] = -y.y * sy;
        }
      }
      group_sync(g);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int u = lt + i * kGT;
        const int a1 = u & 63, blk = (u >> 6) & 7, c = u >> 9;
        const int row = 64 * c + a1;
        store_split8<P>(a_hi, a_lo, off_kmajor(row, kperm(0, 8 * blk)), yre[i]);
        store_split8<P>(a_hi, a_lo, off_kmajor(row, kperm(1, 8 * blk)), yim[i]);
      }
    }
    gemm<P>(g, lt, tmem, ah, al, bh, bl, false, 128, mbar, parity, ok);
    twiddle_to_mn<P, G>(tmem, a_hi, a_lo);
    gemm<P>(g, lt, tmem, ah, al, bh, bl, true, 128, mbar, parity, ok);
    {  // T_b[n1] = wH^(-b n1) conj(D), n1 = n1a + 64 n1b, to the staging columns
      const float2 ta = SM::tin_a()[ttab * 64 + tr];
      const float2 step = SM::tin_b()[ttab * 64 + 1];
      float2* col = SM::col(tslot_);
      const float inv = 1.0f / sy;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float v[32];
        read_chunk(tmem, q, v);
#pragma unroll
        for (int hb = 0; hb < 2; ++hb) {
          const int n1b0 = 32 * th + 16 * q + 8 * hb;
          float2 tw = cmul(ta, SM::tin_b()[ttab * 64 + n1b0]);
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int i = 8 * hb + e;
            const float2 x = make_float2(v[2 * i] * inv, -v[2 * i + 1] * inv);
            col[pad(tr + 64 * (n1b0 + e))] = cmulc(x, tw);
            tw = cmul(tw, step);
          }
        }
      }
    }

    const int64_t krow = k - a.k0;
    if constexpr (kInd) {
      group_sync(g);  // the group's columns and sigma partial are ready
      const float sigma = sqrtf(2.0f * SM::sigpart()[g]) / (float)N;
      if (lt == 0) a.sigma[krow] = sigma;
      combine_and_emit<kF, S, NC, kGT, true>(SM::colptr() + S * g, H, 0, a.kappa * sigma,
                                             (uint32_t)k, krow, out, sigma, lt);
      group_sync(g);  // reads done before the region is overwritten
    } else {
      cluster.sync();  // every column and sigma partial of the cluster is ready
      float tot = 0.f;
#pragma unroll
      for (int q = 0; q < C; ++q) {
        const float* sp = cluster.map_shared_rank(SM::sigpart(), (unsigned)q);
#pragma unroll
        for (int gg = 0; gg < G; ++gg) tot += sp[gg];
      }
      const float sigma = sqrtf(2.0f * tot) / (float)N;
      if (rank == 0 && tid == 0) a.sigma[krow] = sigma;
      combine_and_emit<kF, S, NC, T, true>(SM::colptr(), H, rank, a.kappa * sigma, (uint32_t)k,
                                           krow, out, sigma);
      cluster_sync_after_reads();  // remote reads done before the regions are overwritten
    }
  }

  if (!ok && a.status) atomicOr(a.status, 1u);
  drain_after_give_up(lt, ok, mbar, parity);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot),
                             "r"(128u * G));
}

template <int S, int P, int G>
cudaError_t launch_tc_t(const PlanDev& p, const CorrelateArgs& a, cudaStream_t s) {
  constexpr bool kInd = (S == 2 && G == 2);
  constexpr int C = ColMap<S, kInd ? 2 : 2 * G>::C;
  constexpr size_t smem = TcLay<P, G>::total;
  auto kern = correlate_tc_kernel<S, P, G>;
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
  cfg.blockDim = dim3(kGT * G, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // a kernel that allocates tensor memory runs one CTA per SM
  cfg.gridDim = dim3((unsigned)(sms / C * C), 1, 1);
  int max_clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (max_clusters < 1) return cudaErrorInvalidConfiguration;
  int64_t want = kInd ? (a.k1 - a.k0 + 1) / 2 : a.k1 - a.k0;
  if (a.max_clusters > 0 && want > a.max_clusters) want = a.max_clusters;
  if (want > max_clusters) want = max_clusters;
  cfg.gridDim = dim3((unsigned)(want * C), 1, 1);
  return cudaLaunchKernelEx(&cfg, kern, p, a);
}

}  // namespace tc

cudaError_t launch_correlate_tc(const PlanDev& p, const CorrelateArgs& a, int precision,
                                cudaStream_t s) {
  if (a.k1 <= a.k0) return cudaSuccess;
  const bool bf = precision == 1;
  switch (p.g.S) {
    case 2: return bf ? tc::launch_tc_t<2, tc::BF16X3, 2>(p, a, s) : tc::launch_tc_t<2, tc::FP16X3, 2>(p, a, s);
    case 4: return bf ? tc::launch_tc_t<4, tc::BF16X3, 2>(p, a, s) : tc::launch_tc_t<4, tc::FP16X3, 2>(p, a, s);
    case 8: return bf ? tc::launch_tc_t<8, tc::BF16X3, 2>(p, a, s) : tc::launch_tc_t<8, tc::FP16X3, 2>(p, a, s);
    case 16: return bf ? tc::launch_tc_t<16, tc::BF16X3, 2>(p, a, s) : tc::launch_tc_t<16, tc::FP16X3, 2>(p, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bege
