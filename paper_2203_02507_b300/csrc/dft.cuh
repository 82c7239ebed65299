// Small DFTs held entirely in registers: the butterflies of the tile FFTs.
//
// Products are written with explicit round-to-nearest intrinsics (__fmul_rn,
// __fmaf_rn) so that the compiler cannot contract or reassociate them
// differently in different kernels: every kernel that inlines these helpers
// computes bit-identical results.
//
// Complex additions and subtractions run as one packed FP32x2 instruction on
// the (re, im) pair (add.rn.f32x2 / sub.rn.f32x2, sm_100 and later): the same
// two IEEE operations in one issue slot.  Where a butterfly multiplies by +-i
// the real and imaginary parts trade places, which a packed instruction
// cannot express, so those outputs are written out with scalar operations.
//
// dft<R, S>(v) replaces v[0..R) by X[k] = sum_n v[n] exp(S * 2 pi i n k / R),
// natural order in and out.  S = +1 is the inverse direction (no 1/R factor),
// S = -1 the forward one.  Twiddles inside a DFT are exact constants of the
// mathematics (cos and sin of multiples of pi/8 and pi/6), rounded to float.
#pragma once
#include <cuda_runtime.h>

namespace fpm {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(r)
      : "l"(*reinterpret_cast<const unsigned long long *>(&a)), "l"(*reinterpret_cast<const unsigned long long *>(&b)));
  return *reinterpret_cast<const float2 *>(&r);
}
// a + S i d and a - S i d, part by part (the +-i swaps the parts of d)
template <int S>
__device__ __forceinline__ float2 cadd_si(float2 a, float2 d) {
  return S > 0 ? make_float2(__fsub_rn(a.x, d.y), __fadd_rn(a.y, d.x)) : make_float2(__fadd_rn(a.x, d.y), __fsub_rn(a.y, d.x));
}
template <int S>
__device__ __forceinline__ float2 csub_si(float2 a, float2 d) {
  return S > 0 ? make_float2(__fadd_rn(a.x, d.y), __fsub_rn(a.y, d.x)) : make_float2(__fsub_rn(a.x, d.y), __fadd_rn(a.y, d.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, __fmul_rn(a.y, b.y)), __fmaf_rn(a.y, b.x, -__fmul_rn(a.x, b.y)));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(__fmul_rn(a.x, s), __fmul_rn(a.y, s)); }
// |a|^2
__device__ __forceinline__ float cabs2(float2 a) { return __fmaf_rn(a.x, a.x, __fmul_rn(a.y, a.y)); }
// multiply by S*i
template <int S>
__device__ __forceinline__ float2 mul_si(float2 a) {
  return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// multiply by (c + S i s)
template <int S>
__device__ __forceinline__ float2 mul_cs(float2 a, float c, float s) {
  const float ss = S > 0 ? s : -s;
  return make_float2(__fmaf_rn(a.x, c, -__fmul_rn(a.y, ss)), __fmaf_rn(a.x, ss, __fmul_rn(a.y, c)));
}

// cos(pi/8), sin(pi/8), sqrt(1/2), sqrt(3)/2
#define FPM_C8 0.92387953251128674f
#define FPM_S8 0.38268343236508977f
#define FPM_R2 0.70710678118654752f
#define FPM_R3 0.86602540378443865f

template <int S>
__device__ __forceinline__ void dft2(float2 &a, float2 &b) {
  const float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <int S>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
  const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
  const float2 t2 = cadd(a1, a3), d = csub(a1, a3);
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd_si<S>(t1, d);     // t1 + S i d
  a3 = csub_si<S>(t1, d);     // t1 - S i d
}

// X[k] = sum v[n] w^{nk}, w = exp(S 2 pi i / 3)
template <int S>
__device__ __forceinline__ void dft3(float2 &a0, float2 &a1, float2 &a2) {
  const float2 s = cadd(a1, a2);
  const float2 d = mul_si<S>(csub(a1, a2));     // S i (a1 - a2)
  const float2 m = make_float2(__fmaf_rn(-0.5f, s.x, a0.x), __fmaf_rn(-0.5f, s.y, a0.y));
  a0 = cadd(a0, s);
  a1 = make_float2(__fmaf_rn(FPM_R3, d.x, m.x), __fmaf_rn(FPM_R3, d.y, m.y));
  a2 = make_float2(__fmaf_rn(-FPM_R3, d.x, m.x), __fmaf_rn(-FPM_R3, d.y, m.y));
}

template <int R, int S>
struct Dft;

template <int S>
struct Dft<2, S> {
  __device__ __forceinline__ static void run(float2 *v) { dft2<S>(v[0], v[1]); }
};

template <int S>
struct Dft<4, S> {
  __device__ __forceinline__ static void run(float2 *v) { dft4<S>(v[0], v[1], v[2], v[3]); }
};

template <int S>
struct Dft<3, S> {
  __device__ __forceinline__ static void run(float2 *v) { dft3<S>(v[0], v[1], v[2]); }
};

// 8 = 2 x 4: even/odd halves, then one radix-2 stage with w8^k
template <int S>
struct Dft<8, S> {
  __device__ __forceinline__ static void run(float2 *v) {
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<S>(e0, e1, e2, e3);
    dft4<S>(o0, o1, o2, o3);
    o1 = mul_cs<S>(o1, FPM_R2, FPM_R2);
    o3 = mul_cs<S>(o3, -FPM_R2, FPM_R2);
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd_si<S>(e2, o2);  // e2 + S i o2
    v[6] = csub_si<S>(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
  }
};

// 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2
template <int S>
struct Dft<16, S> {
  __device__ __forceinline__ static void run(float2 *v) {
    float2 y[16];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      float2 a0 = v[n2], a1 = v[4 + n2], a2 = v[8 + n2], a3 = v[12 + n2];
      dft4<S>(a0, a1, a2, a3);                 // a_k1
      y[n2 * 4 + 0] = a0;
      y[n2 * 4 + 1] = a1;
      y[n2 * 4 + 2] = a2;
      y[n2 * 4 + 3] = a3;
    }
    // twiddles w16^{n2 k1}
    y[1 * 4 + 1] = mul_cs<S>(y[5], FPM_C8, FPM_S8);    // w^1
    y[1 * 4 + 2] = mul_cs<S>(y[6], FPM_R2, FPM_R2);    // w^2
    y[1 * 4 + 3] = mul_cs<S>(y[7], FPM_S8, FPM_C8);    // w^3
    y[2 * 4 + 1] = mul_cs<S>(y[9], FPM_R2, FPM_R2);    // w^2
    y[2 * 4 + 2] = mul_si<S>(y[10]);                   // w^4
    y[2 * 4 + 3] = mul_cs<S>(y[11], -FPM_R2, FPM_R2);  // w^6
    y[3 * 4 + 1] = mul_cs<S>(y[13], FPM_S8, FPM_C8);   // w^3
    y[3 * 4 + 2] = mul_cs<S>(y[14], -FPM_R2, FPM_R2);  // w^6
    y[3 * 4 + 3] = mul_cs<S>(y[15], -FPM_C8, -FPM_S8); // w^9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      float2 a0 = y[k1], a1 = y[4 + k1], a2 = y[8 + k1], a3 = y[12 + k1];
      dft4<S>(a0, a1, a2, a3);                 // over n2 -> k2
      v[k1] = a0;
      v[k1 + 4] = a1;
      v[k1 + 8] = a2;
      v[k1 + 12] = a3;
    }
  }
};

// 12 = 3 x 4: n = 4 n1 + n2 (n1 < 3, n2 < 4), k = k1 + 3 k2
template <int S>
struct Dft<12, S> {
  __device__ __forceinline__ static void run(float2 *v) {
    float2 y[12];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      float2 a0 = v[n2], a1 = v[4 + n2], a2 = v[8 + n2];
      dft3<S>(a0, a1, a2);
      y[n2 * 3 + 0] = a0;
      y[n2 * 3 + 1] = a1;
      y[n2 * 3 + 2] = a2;
    }
    // twiddles w12^{n2 k1}: w^1 = (r3, S/2), w^2 = (1/2, S r3), w^3 = S i, w^4 = (-1/2, S r3), w^6 = -1
    y[1 * 3 + 1] = mul_cs<S>(y[4], FPM_R3, 0.5f);
    y[1 * 3 + 2] = mul_cs<S>(y[5], 0.5f, FPM_R3);
    y[2 * 3 + 1] = mul_cs<S>(y[7], 0.5f, FPM_R3);
    y[2 * 3 + 2] = mul_cs<S>(y[8], -0.5f, FPM_R3);
    y[3 * 3 + 1] = mul_si<S>(y[10]);
    y[3 * 3 + 2] = make_float2(-y[11].x, -y[11].y);
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
      float2 a0 = y[k1], a1 = y[3 + k1], a2 = y[6 + k1], a3 = y[9 + k1];
      dft4<S>(a0, a1, a2, a3);
      v[k1] = a0;
      v[k1 + 3] = a1;
      v[k1 + 6] = a2;
      v[k1 + 9] = a3;
    }
  }
};

// dft4 of inputs of which only those in IN (bit i: a_i may be nonzero; the
// others are exactly zero) and outputs of which only those in OUT are needed
// (the others are left unspecified).  Every needed output is computed with the
// operations of dft4<S> in the same order, minus the additions of zeros, so it
// equals dft4<S>'s output (an exact-zero result may differ in its sign).
template <int S, int IN, int OUT>
__device__ __forceinline__ void dft4_band(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
  constexpr bool i0 = IN & 1, i1 = IN & 2, i2 = IN & 4, i3 = IN & 8;
  static_assert((i0 || i2) && (i1 || i3), "each half of the butterfly has a nonzero input");
  auto neg = [](float2 z) { return make_float2(-z.x, -z.y); };
  const float2 t0 = (i0 && i2) ? cadd(a0, a2) : i0 ? a0 : a2;
  const float2 t1 = (i0 && i2) ? csub(a0, a2) : i0 ? a0 : neg(a2);
  const float2 t2 = (i1 && i3) ? cadd(a1, a3) : i1 ? a1 : a3;
  const float2 d = (i1 && i3) ? csub(a1, a3) : i1 ? a1 : neg(a3);
  if constexpr ((OUT & 1) != 0) a0 = cadd(t0, t2);
  if constexpr ((OUT & 4) != 0) a2 = csub(t0, t2);
  if constexpr ((OUT & 2) != 0) a1 = cadd_si<S>(t1, d);
  if constexpr ((OUT & 8) != 0) a3 = csub_si<S>(t1, d);
}

// Dft<16, S> for inputs that are zero outside [ILO, IHI] and outputs needed only
// in [OLO, OHI] (a band of the line: the support of a disc in the middle of the
// box).  The same butterflies, twiddles and order as Dft<16, S>, so the needed
// outputs are its outputs; additions of the known zeros and the butterflies of
// unneeded outputs are left out at compile time.
template <int S, int ILO, int IHI, int OLO, int OHI>
struct DftBand16 {
  template <int N2>
  static constexpr int in_mask() {
    return ((N2 >= ILO && N2 <= IHI) ? 1 : 0) | ((N2 + 4 >= ILO && N2 + 4 <= IHI) ? 2 : 0) |
           ((N2 + 8 >= ILO && N2 + 8 <= IHI) ? 4 : 0) | ((N2 + 12 >= ILO && N2 + 12 <= IHI) ? 8 : 0);
  }
  template <int K1>
  static constexpr int out_mask() {
    return ((K1 >= OLO && K1 <= OHI) ? 1 : 0) | ((K1 + 4 >= OLO && K1 + 4 <= OHI) ? 2 : 0) |
           ((K1 + 8 >= OLO && K1 + 8 <= OHI) ? 4 : 0) | ((K1 + 12 >= OLO && K1 + 12 <= OHI) ? 8 : 0);
  }
  template <int N2>
  __device__ __forceinline__ static void stage1(const float2 *v, float2 *y) {
    float2 a0 = v[N2], a1 = v[4 + N2], a2 = v[8 + N2], a3 = v[12 + N2];
    dft4_band<S, in_mask<N2>(), 15>(a0, a1, a2, a3);
    y[N2 * 4 + 0] = a0;
    y[N2 * 4 + 1] = a1;
    y[N2 * 4 + 2] = a2;
    y[N2 * 4 + 3] = a3;
  }
  template <int K1>
  __device__ __forceinline__ static void stage2(const float2 *y, float2 *v) {
    constexpr int om = out_mask<K1>();
    if constexpr (om != 0) {
      float2 a0 = y[K1], a1 = y[4 + K1], a2 = y[8 + K1], a3 = y[12 + K1];
      dft4_band<S, 15, om>(a0, a1, a2, a3);
      if constexpr ((om & 1) != 0) v[K1] = a0;
      if constexpr ((om & 2) != 0) v[K1 + 4] = a1;
      if constexpr ((om & 4) != 0) v[K1 + 8] = a2;
      if constexpr ((om & 8) != 0) v[K1 + 12] = a3;
    }
  }
  __device__ __forceinline__ static void run(float2 *v) {
    float2 y[16];
    stage1<0>(v, y);
    stage1<1>(v, y);
    stage1<2>(v, y);
    stage1<3>(v, y);
    // twiddles w16^{n2 k1}, as in Dft<16, S>
    y[1 * 4 + 1] = mul_cs<S>(y[5], FPM_C8, FPM_S8);    // w^1
    y[1 * 4 + 2] = mul_cs<S>(y[6], FPM_R2, FPM_R2);    // w^2
    y[1 * 4 + 3] = mul_cs<S>(y[7], FPM_S8, FPM_C8);    // w^3
    y[2 * 4 + 1] = mul_cs<S>(y[9], FPM_R2, FPM_R2);    // w^2
    y[2 * 4 + 2] = mul_si<S>(y[10]);                   // w^4
    y[2 * 4 + 3] = mul_cs<S>(y[11], -FPM_R2, FPM_R2);  // w^6
    y[3 * 4 + 1] = mul_cs<S>(y[13], FPM_S8, FPM_C8);   // w^3
    y[3 * 4 + 2] = mul_cs<S>(y[14], -FPM_R2, FPM_R2);  // w^6
    y[3 * 4 + 3] = mul_cs<S>(y[15], -FPM_C8, -FPM_S8); // w^9
    stage2<0>(y, v);
    stage2<1>(y, v);
    stage2<2>(y, v);
    stage2<3>(y, v);
  }
};

}  // namespace fpm
