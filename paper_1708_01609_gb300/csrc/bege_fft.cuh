// Register-level DFT kernels and shared-memory Stockham passes for the
// column FFTs of the correlation (Eq. 3S).  Forward kernel exp(-i ...) as in
// Eq. A2; the inverse uses exp(+i ...) without the 1/N factor.
#pragma once

#include <cuda_runtime.h>

namespace bege {

// Shared-memory index with one padding slot every 16 complex values: keeps
// the strided Stockham stores (stride 16 and 17*16) free of bank conflicts.
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

template <int F>
__host__ __device__ constexpr int col_stride() { return F + F / 16; }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// a * b
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

constexpr float kC1 = 0.92387953251128674f;  // cos(pi/8)
constexpr float kS1 = 0.38268343236508978f;  // sin(pi/8)
constexpr float kR2 = 0.70710678118654752f;  // cos(pi/4)
constexpr float kT1 = 0.41421356237309505f;  // tan(pi/8)

// Twiddles in factored form, so that a twiddle multiply and the addition
// that follows it become fused multiply-adds (the tangent form of a
// rotation: exp(-i a) = cos a (1 - i tan a)).  rot_a multiplies by
// (1 - i t) in the forward direction and (1 + i t) in the inverse one (the
// direction of w16 = exp(-i pi/8) and of its conjugate); rot_b the opposite.
template <bool INV>
__device__ __forceinline__ float2 rot_a(float2 q, float t) {
  return INV ? make_float2(fmaf(-t, q.y, q.x), fmaf(t, q.x, q.y))
             : make_float2(fmaf(t, q.y, q.x), fmaf(-t, q.x, q.y));
}
template <bool INV>
__device__ __forceinline__ float2 rot_b(float2 q, float t) {
  return rot_a<!INV>(q, t);
}
// t = 1: (1 -/+ i) q with two additions
template <bool INV>
__device__ __forceinline__ float2 rot_a1(float2 q) {
  return INV ? make_float2(q.x - q.y, q.y + q.x) : make_float2(q.x + q.y, q.y - q.x);
}
template <bool INV>
__device__ __forceinline__ float2 rot_b1(float2 q) {
  return rot_a1<!INV>(q);
}
// p + s u, componentwise
__device__ __forceinline__ float2 cfma(float2 p, float s, float2 u) {
  return make_float2(fmaf(s, u.x, p.x), fmaf(s, u.y, p.y));
}

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// In place, natural order in and out.
template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 s02 = cadd(x0, x2), d02 = csub(x0, x2);
  float2 s13 = cadd(x1, x3), d13 = mul_mi<INV>(csub(x1, x3));
  x0 = cadd(s02, s13);
  x2 = csub(s02, s13);
  x1 = cadd(d02, d13);
  x3 = csub(d02, d13);
}

// DFT4 of (x0, w x1, w^2 x2, w^3 x3) with w = w16^K1 (forward) or its
// conjugate (inverse), in place, natural order out.  With a = x0 + w^2 x2,
// b = x0 - w^2 x2, c = x1 + w^2 x3, d = x1 - w^2 x3 the outputs are
// a + w c, b + m(w d), a - w c, b - m(w d), m = multiplication by -i
// (forward) or +i (inverse); each twiddle enters through the tangent form,
// so a twiddle multiply and its addition cost two fused multiply-adds.
template <bool INV, int K1>
__device__ __forceinline__ void dft4_tw16(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 a, b, c, d;
  if constexpr (K1 == 0) {
    dft4<INV>(x0, x1, x2, x3);
    return;
  } else if constexpr (K1 == 1) {  // w^2 = w8 = r2 (1 -/+ i)
    const float2 u2 = rot_a1<INV>(x2), u3 = rot_a1<INV>(x3);
    a = cfma(x0, kR2, u2); b = cfma(x0, -kR2, u2);
    c = cfma(x1, kR2, u3); d = cfma(x1, -kR2, u3);
    // w = c1 (1 -/+ i t1)
    const float2 vc = rot_a<INV>(c, kT1), vd = mul_mi<INV>(rot_a<INV>(d, kT1));
    x0 = cfma(a, kC1, vc); x2 = cfma(a, -kC1, vc);
    x1 = cfma(b, kC1, vd); x3 = cfma(b, -kC1, vd);
  } else if constexpr (K1 == 2) {  // w^2 = w4 = m, w = w8 = r2 (1 -/+ i)
    const float2 m2 = mul_mi<INV>(x2), m3 = mul_mi<INV>(x3);
    a = cadd(x0, m2); b = csub(x0, m2);
    c = cadd(x1, m3); d = csub(x1, m3);
    const float2 uc = rot_a1<INV>(c), ud = mul_mi<INV>(rot_a1<INV>(d));
    x0 = cfma(a, kR2, uc); x2 = cfma(a, -kR2, uc);
    x1 = cfma(b, kR2, ud); x3 = cfma(b, -kR2, ud);
  } else {  // K1 == 3: w^2 = w8^3 = -r2 (1 +/- i), w = w16^3 = m(c1 (1 +/- i t1))
    static_assert(K1 == 3, "twiddle index");
    const float2 u2 = rot_b1<INV>(x2), u3 = rot_b1<INV>(x3);
    a = cfma(x0, -kR2, u2); b = cfma(x0, kR2, u2);
    c = cfma(x1, -kR2, u3); d = cfma(x1, kR2, u3);
    // w c = m(c1 vc); m(w d) = m(m(c1 vd)) = -c1 vd
    const float2 vc = mul_mi<INV>(rot_b<INV>(c, kT1)), vd = rot_b<INV>(d, kT1);
    x0 = cfma(a, kC1, vc); x2 = cfma(a, -kC1, vc);
    x1 = cfma(b, -kC1, vd); x3 = cfma(b, kC1, vd);
  }
}

template <bool INV>
__device__ __forceinline__ void dft8(float2 (&x)[8]) {
  float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  float2 o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  // e_k +/- w8^k o_k: w8 = r2 (1 -/+ i), w8^2 = m, w8^3 = -r2 (1 +/- i)
  const float2 u1 = rot_a1<INV>(o1), u3 = rot_b1<INV>(o3);
  o2 = mul_mi<INV>(o2);
  x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
  x[1] = cfma(e1, kR2, u1); x[5] = cfma(e1, -kR2, u1);
  x[2] = cadd(e2, o2); x[6] = csub(e2, o2);
  x[3] = cfma(e3, -kR2, u3); x[7] = cfma(e3, kR2, u3);
}

// 16 = 4 x 4: DFT4 over the stride-4 index, twiddle w16^(n2 k1), DFT4 over
// the offset index, then transpose to natural order.  HALFZ: inputs 8..15
// are known to be zero (a zero-padded half), which shortens the first DFT4s.
template <bool INV, bool HALFZ = false>
__device__ __forceinline__ void dft16(float2 (&x)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    if constexpr (HALFZ) {
      const float2 a = x[n2], b = x[n2 + 4];
      const float2 mb = mul_mi<INV>(b);
      x[n2] = cadd(a, b);
      x[n2 + 8] = csub(a, b);
      x[n2 + 4] = cadd(a, mb);
      x[n2 + 12] = csub(a, mb);
    } else {
      dft4<INV>(x[n2], x[n2 + 4], x[n2 + 8], x[n2 + 12]);
    }
  }
  // DFT4 over n2 of x[n2 + 4 k1] w16^(n2 k1), the twiddles merged into it
  dft4_tw16<INV, 0>(x[0], x[1], x[2], x[3]);
  dft4_tw16<INV, 1>(x[4], x[5], x[6], x[7]);
  dft4_tw16<INV, 2>(x[8], x[9], x[10], x[11]);
  dft4_tw16<INV, 3>(x[12], x[13], x[14], x[15]);
  float2 t[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = x[4 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = t[i];
}

template <int R, bool INV, bool HALFZ = false>
__device__ __forceinline__ void dft(float2 (&x)[R]) {
  static_assert(!HALFZ || R == 16, "half-zero DFT only for radix 16");
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2<INV>(x[0], x[1]);
  } else if constexpr (R == 4) {
    dft4<INV>(x[0], x[1], x[2], x[3]);
  } else if constexpr (R == 8) {
    dft8<INV>(x);
  } else {
    static_assert(R == 16, "radix");
    dft16<INV, HALFZ>(x);
  }
}

// One in-place Stockham pass of radix R over NC columns of length F in
// shared memory (column c at cols + c * col_stride<F>(), padded indexing).
// Butterfly j reads col[j + r F/R], twiddles by w(NS R)^(k r) with
// k = j mod NS (table tw[r*NS + k]), and writes col[(j-k) R + k + r NS].
// Butterflies are taken in rounds of T threads; since F/R divides T every
// round covers whole columns, so a round can load, synchronise and store
// without touching the columns of the next round.  Each thread holds one
// butterfly (R complex values) across a barrier: holding two (one round)
// costs fewer barriers but spills at 128 registers and measured slower.
// With F/R and NS multiples of 16 the padded addresses of a butterfly are
// one base plus constants.
template <int F, int NC, int T, int R, int NS, bool INV, bool TRAIL = true>
__device__ __forceinline__ void stockham_pass(float2* cols, const float2* tw) {
  constexpr int NB = F / R;
  static_assert(T % NB == 0, "rounds must cover whole columns");
  constexpr int total = NC * NB;
  constexpr int rounds = (total + T - 1) / T;
  constexpr int CS = col_stride<F>();
#pragma unroll
  for (int i = 0; i < rounds; ++i) {
    const int idx = threadIdx.x + i * T;
    const bool act = (total % T == 0) || idx < total;
    const int c = idx / NB, j = idx - c * NB;
    const int k = j & (NS - 1);
    float2 v[R];
    if (act) {
      const float2* col = cols + c * CS;
      if constexpr (NB % 16 == 0) {
        const float2* p = col + pad(j);
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = p[r * (NB + NB / 16)];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = col[pad(j + r * NB)];
      }
      if constexpr (NS > 1) {
        const float2* t = tw + k;
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = INV ? cmulc(v[r], t[r * NS]) : cmul(v[r], t[r * NS]);
      }
      dft<R, INV>(v);
    }
    __syncthreads();
    if (act) {
      float2* col = cols + c * CS;
      const int base = (j - k) * R + k;
      if constexpr (NS % 16 == 0) {
        float2* p = col + pad(base);
#pragma unroll
        for (int r = 0; r < R; ++r) p[r * (NS + NS / 16)] = v[r];
      } else if constexpr (NS == 1 && R == 16) {
        float2* p = col + pad(base);
#pragma unroll
        for (int r = 0; r < R; ++r) p[r] = v[r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) col[pad(base + r * NS)] = v[r];
      }
    }
  }
  // TRAIL = false: the caller's next pass runs the same rounds over the same
  // columns, so with two or more rounds each column's stores here and its
  // loads there are separated by a later round's barrier (of this pass or
  // of the next); with one round they are not, and the barrier stays
  if constexpr (TRAIL || rounds < 2) __syncthreads();
}

}  // namespace bege
