// Precision form: the column FFTs of the correlation on the 5th-generation
// tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// Every 4096-point column transform is a four-step of 64 x 64:
//   V[m1][k1] = sum_{m2} u[m1 + 64 m2] w64^(m2 k1)          (GEMM 1)
//   V'        = V[m1][k1] w4096^(m1 k1)                       (FP32 twiddle)
//   Z[k1 + 64 k2] = sum_{m1} V'[m1][k1] w64^(m1 k2)           (GEMM 2)
// A group of 8 warps holds the two columns of a unit (b, S-b), so each GEMM
// is [128 rows] x [128 real K] x [128 real N]: complex values as (re, im)
// pairs, the 64-point DFT matrix as real 2 x 2 blocks.  A kernel that
// allocates tensor memory runs one CTA per SM, so a CTA carries G = 2 groups
// (two units, 512 threads) where the transform has S >= 4 columns: each
// group has its own operands, accumulator (128 TMEM columns) and mbarrier,
// synchronises on its own named barrier, and one group's MMAs overlap the
// other's CUDA-core work.  The inverse
// transform reuses the forward one, IDFT(Y) = conj(DFT(conj(Y))).
// Operands are split into a high and a low 16-bit part and the GEMM is a sum
// of products of parts, accumulated in FP32:
//   BF16x3: A_hi B_hi + A_lo B_hi + A_hi B_lo
//   FP16x3: the same three products in FP16 (three more mantissa bits than
//           BF16, far less range: each transform's input is scaled by a power
//           of two into FP16's range and the output scaled back, exactly)
// Two terms (an FP16 DFT matrix without its low part) are not enough: on
// narrowband chirps its rounding alone exceeds 2e-3 sigma.
// Twiddles, the spectral product, the Parseval sum and the S-point combine
// stay in FP32 (the single-segment kernel's arithmetic).
//
// Shared-memory operands use the no-swizzle canonical layout: core matrices
// of 8 rows x 16 bytes; K-major for GEMM 1 (rows are the column rows, K the
// transform input) and MN-major for GEMM 2 (written straight from the rows
// of the GEMM-1 accumulator, so no transpose pass is needed).  One thread per group
// issues the MMAs; completion is signalled through an mbarrier whose wait is
// bounded (on give-up the kernel flags `status` and carries on, so every
// barrier is still reached and tensor memory is freed).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "bege_corr.cuh"

namespace bege {
namespace tc {

constexpr int kF = 4096;
constexpr int kGT = 256;  // threads of a group: 8 warps, two per TMEM lane quarter

enum { FP16X3 = 0, BF16X3 = 1 };

template <int P>
struct Part;
template <>
struct Part<FP16X3> {
  using T = __half;
  static constexpr uint32_t fmt = 0;
  static constexpr int terms = 3;
  static __device__ __forceinline__ T cvt(float x) { return __float2half_rn(x); }
  static __device__ __forceinline__ float back(T h) { return __half2float(h); }
};
template <>
struct Part<BF16X3> {
  using T = __nv_bfloat16;
  static constexpr uint32_t fmt = 1;
  static constexpr int terms = 3;
  static __device__ __forceinline__ T cvt(float x) { return __float2bfloat16_rn(x); }
  static __device__ __forceinline__ float back(T h) { return __bfloat162float(h); }
};

// Shared-memory layout (bytes) for G groups of 8 warps, group g holding
// column slots 2g, 2g+1.  A group's FP32 staging columns and its 16-bit A
// operand share one region: A is live from a transform's first operand build
// to the completion of its second GEMM, the columns from there to the end of
// the product (forward) or of the combine (inverse).  The DFT matrix and the
// twiddle tables are shared by the groups.
template <int P, int G>
struct TcLay {
  static constexpr int CS = col_stride<kF>();
  static constexpr size_t R = 2 * CS * 8;                           // one group's region
  static_assert(R >= 65536 && R % 128 == 0, "region holds A_hi and A_lo");
  static constexpr size_t cols = 0;                                 // slot s at s * CS float2
  static constexpr size_t b_hi = G * R;                             // 128 x 128 16-bit
  static constexpr size_t b_lo = b_hi + 32768;
  static constexpr size_t w64 = b_lo + 32768;                       // w64^k, k < 64
  static constexpr size_t w4k = w64 + 64 * 8;                       // w4096^k, k < 64
  static constexpr size_t tin_a = w4k + 64 * 8;                     // [slot][x] wH^(b x)
  static constexpr size_t tin_b = tin_a + 2 * G * 64 * 8;           // [slot][x] wH^(64 b x)
  static constexpr size_t colptr = tin_b + 2 * G * 64 * 8;
  static constexpr size_t red = colptr + 16 * 8;                    // [group][32]
  static constexpr size_t sigpart = red + G * 32 * 4;               // [group]
  static constexpr size_t mbar = sigpart + 16;                      // [group]
  static constexpr size_t tslot = mbar + 8 * G;
  static constexpr size_t total = tslot + 8;
  static __host__ __device__ constexpr size_t a_hi(int g) { return g * R; }
  static __host__ __device__ constexpr size_t a_lo(int g) { return g * R + 32768; }
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// K index of (part, x): the 32 lowest x first, so a half-zero input (x < 32)
// occupies K < 64.
__device__ __forceinline__ int kperm(int part, int x) { return (x >> 5) * 64 + part * 32 + (x & 31); }

// Byte offsets of element (row, K) of a 128 x 128 16-bit operand.
__device__ __forceinline__ uint32_t off_kmajor(int row, int k) {
  return (row >> 3) * 2048 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ uint32_t off_mnmajor(int row, int k) {
  return (row >> 3) * 128 + (k >> 3) * 2048 + (k & 7) * 16 + (row & 7) * 2;
}

// tcgen05 shared-memory matrix descriptor, no swizzle: start address, LBO
// (byte stride between core matrices along K), SBO (along M/N), fixed 0b001.
__device__ __forceinline__ uint64_t mdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulate, A/B format, A major,
// B K-major, N = 128, M = 128.
__device__ __forceinline__ uint32_t idesc(uint32_t fmt, bool a_mn_major) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((a_mn_major ? 1u : 0u) << 15) |
         ((128u >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t id,
                                        uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(id), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 20) && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
  }
  return done != 0;
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Split 8 FP32 values into their high and low 16-bit parts, hi = rn(x),
// lo = rn(x - hi), converting two values per instruction, and store each
// part as one 16-byte run (8 consecutive K or rows).
template <int P>
__device__ __forceinline__ void store_split8(unsigned char* hi, unsigned char* lo, uint32_t off,
                                             const float (&x)[8]) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if constexpr (P == FP16X3) {
      const __half2 hh = __floats2half2_rn(x[2 * e], x[2 * e + 1]);
      const float2 bk = __half22float2(hh);
      const __half2 ll = __floats2half2_rn(x[2 * e] - bk.x, x[2 * e + 1] - bk.y);
      h[e] = *reinterpret_cast<const uint32_t*>(&hh);
      l[e] = *reinterpret_cast<const uint32_t*>(&ll);
    } else {
      const __nv_bfloat162 hh = __floats2bfloat162_rn(x[2 * e], x[2 * e + 1]);
      const float2 bk = __bfloat1622float2(hh);
      const __nv_bfloat162 ll = __floats2bfloat162_rn(x[2 * e] - bk.x, x[2 * e + 1] - bk.y);
      h[e] = *reinterpret_cast<const uint32_t*>(&hh);
      l[e] = *reinterpret_cast<const uint32_t*>(&ll);
    }
  }
  *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

template <int P, int G>
struct Smem {
  using L = TcLay<P, G>;
  static __device__ __forceinline__ float2* col(int slot) {
    return reinterpret_cast<float2*>(smem_raw + L::cols) + slot * L::CS;
  }
  static __device__ __forceinline__ float2* w64() { return reinterpret_cast<float2*>(smem_raw + L::w64); }
  static __device__ __forceinline__ float2* w4k() { return reinterpret_cast<float2*>(smem_raw + L::w4k); }
  static __device__ __forceinline__ float2* tin_a() { return reinterpret_cast<float2*>(smem_raw + L::tin_a); }
  static __device__ __forceinline__ float2* tin_b() { return reinterpret_cast<float2*>(smem_raw + L::tin_b); }
  static __device__ __forceinline__ float2** colptr() { return reinterpret_cast<float2**>(smem_raw + L::colptr); }
  static __device__ __forceinline__ float* red(int g) { return reinterpret_cast<float*>(smem_raw + L::red) + 32 * g; }
  static __device__ __forceinline__ float* sigpart() { return reinterpret_cast<float*>(smem_raw + L::sigpart); }
};

__device__ __forceinline__ float2 root(int64_t k, int64_t M) {
  double s, c;
  sincospi(-2.0 * (double)(k % M) / (double)M, &s, &c);
  return make_float2((float)c, (float)s);
}

// w4096^p for p < 4096 from the two 64-entry tables: w64^(p/64) w4096^(p%64).
template <int P, int G>
__device__ __forceinline__ float2 w4096(int p) {
  return cmul(Smem<P, G>::w64()[p >> 6], Smem<P, G>::w4k()[p & 63]);
}

// Issue one GEMM: D = sum of the part products over K (K = 64 or 128), then
// commit to the mbarrier.  One thread of the group.  ah, al: the group's A
// parts; bh, bl: the DFT matrix parts (shared-memory addresses).
template <int P>
__device__ __forceinline__ void issue_gemm(uint32_t tmem, uint32_t ah, uint32_t al, uint32_t bh,
                                           uint32_t bl, bool a_mn, int K, uint32_t mbar) {
  // K-major A: LBO 128 (along K), SBO 2048 (along rows); MN-major A: LBO 2048, SBO 128
  const uint32_t a_lbo = a_mn ? 2048u : 128u, a_sbo = a_mn ? 128u : 2048u;
  const uint32_t a_step = a_mn ? 4096u : 256u;  // 16 K = two core matrices along K
  const uint32_t id = idesc(Part<P>::fmt, a_mn);
  uint32_t acc = 0;
  for (int t = 0; t < Part<P>::terms; ++t) {
    const uint32_t a0 = (t == 1) ? al : ah;
    const uint32_t b0 = (t == 2) ? bl : bh;
    for (int kk = 0; kk < K / 16; ++kk) {
      mma_f16(tmem, mdesc(a0 + kk * a_step, a_lbo, a_sbo), mdesc(b0 + kk * 256, 128, 2048), id,
              acc);
      acc = 1;
    }
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      mbar));
}

}  // namespace tc
}  // namespace bege
