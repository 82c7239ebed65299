// Small DFTs on two independent transforms at once, with packed FP32x2 arithmetic.
//
// sm_100-class GPUs execute add/sub/mul/fma on a pair of FP32 values as one
// instruction (`add.rn.f32x2` and friends; FADD2/FMUL2/FFMA2): the pair goes
// through the FMA pipe at the scalar rate per value, but takes one issue slot
// instead of two.  The fused update is bound by instruction issue as much as
// by FP32 throughput, so its butterflies run on such pairs: a lane holds the
// same element of two transforms (two rows, or two columns, of one update) as
// a `cpair` {re = (re0, re1), im = (im0, im1)} and every butterfly step is one
// packed instruction for both.
//
// Every value is computed with exactly the scalar operations of dft.cuh
// (same order, same rounding: x - y and x + (-y) are the same IEEE operation,
// and -(a*b) == a*(-b)), so a transform computed here equals, bit for bit,
// the same transform computed with the scalar helpers.
#pragma once
#include <cuda_runtime.h>

#include "dft.cuh"

namespace fpm {

struct cpair {
  float2 re, im;   // (transform 0, transform 1)
};

__device__ __forceinline__ float2 p2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p2sub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(r)
      : "l"(*reinterpret_cast<const unsigned long long *>(&a)), "l"(*reinterpret_cast<const unsigned long long *>(&b)));
  return *reinterpret_cast<const float2 *>(&r);
}
__device__ __forceinline__ float2 p2dup(float v) { return make_float2(v, v); }
// exact negation of both halves
__device__ __forceinline__ float2 p2neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ cpair cpzero() { return cpair{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
__device__ __forceinline__ cpair cpadd(cpair a, cpair b) { return cpair{p2add(a.re, b.re), p2add(a.im, b.im)}; }
__device__ __forceinline__ cpair cpsub(cpair a, cpair b) { return cpair{p2sub(a.re, b.re), p2sub(a.im, b.im)}; }
// a * w for one complex w shared by both transforms, given as the pairs
// (w.x, w.x), (w.y, w.y) and (-w.y, -w.y): same operations as cmul(a, w)
__device__ __forceinline__ cpair cpmul_w(cpair a, float2 wx, float2 wy, float2 nwy) {
  return cpair{p2fma(a.re, wx, p2mul(a.im, nwy)), p2fma(a.re, wy, p2mul(a.im, wx))};
}
// a * b per transform: same operations as cmul
__device__ __forceinline__ cpair cpmul(cpair a, cpair b) {
  return cpair{p2fma(a.re, b.re, p2neg(p2mul(a.im, b.im))), p2fma(a.re, b.im, p2mul(a.im, b.re))};
}
// a * conj(b) per transform: same operations as cmulc
__device__ __forceinline__ cpair cpmulc(cpair a, cpair b) {
  return cpair{p2fma(a.re, b.re, p2mul(a.im, b.im)), p2fma(a.im, b.re, p2neg(p2mul(a.re, b.im)))};
}
__device__ __forceinline__ cpair cpscale(cpair a, float2 s) { return cpair{p2mul(a.re, s), p2mul(a.im, s)}; }
// |a|^2 per transform: same operations as cabs2
__device__ __forceinline__ float2 cpabs2(cpair a) { return p2fma(a.re, a.re, p2mul(a.im, a.im)); }
// multiply by (c + S i s), c and s compile-time constants: same operations as
// mul_cs, on each half with scalar instructions whose constant operand is an
// immediate (a packed instruction would need the constant pair in registers)
template <int S>
__device__ __forceinline__ cpair cpmul_cs(cpair a, float c, float s) {
  const float ss = S > 0 ? s : -s;
  cpair r;
  r.re.x = __fmaf_rn(a.re.x, c, __fmul_rn(a.im.x, -ss));
  r.re.y = __fmaf_rn(a.re.y, c, __fmul_rn(a.im.y, -ss));
  r.im.x = __fmaf_rn(a.re.x, ss, __fmul_rn(a.im.x, c));
  r.im.y = __fmaf_rn(a.re.y, ss, __fmul_rn(a.im.y, c));
  return r;
}
// multiply by S*i: a pure exchange of halves with one sign flip; callers fold
// it into the next add or subtract instead (see dft4p)
template <int S>
__device__ __forceinline__ cpair cpmul_si(cpair a) {
  return S > 0 ? cpair{p2neg(a.im), a.re} : cpair{a.im, p2neg(a.re)};
}

template <int S>
__device__ __forceinline__ void dft2p(cpair &a, cpair &b) {
  const cpair t = a;
  a = cpadd(t, b);
  b = cpsub(t, b);
}

// dft4 with the multiplication by S*i folded into the last adds and subtracts:
// t1 + S i d = (t1.re - S d.im, t1.im + S d.re)
template <int S>
__device__ __forceinline__ void dft4p(cpair &a0, cpair &a1, cpair &a2, cpair &a3) {
  const cpair t0 = cpadd(a0, a2), t1 = cpsub(a0, a2);
  const cpair t2 = cpadd(a1, a3), d = cpsub(a1, a3);
  a0 = cpadd(t0, t2);
  a2 = cpsub(t0, t2);
  if (S > 0) {
    a1 = cpair{p2sub(t1.re, d.im), p2add(t1.im, d.re)};
    a3 = cpair{p2add(t1.re, d.im), p2sub(t1.im, d.re)};
  } else {
    a1 = cpair{p2add(t1.re, d.im), p2sub(t1.im, d.re)};
    a3 = cpair{p2sub(t1.re, d.im), p2add(t1.im, d.re)};
  }
}

// X[k] = sum v[n] w^{nk}, w = exp(S 2 pi i / 3); same steps as dft3
template <int S>
__device__ __forceinline__ void dft3p(cpair &a0, cpair &a1, cpair &a2) {
  const cpair s = cpadd(a1, a2);
  const cpair d0 = cpsub(a1, a2);
  // d = S i d0
  const cpair d = S > 0 ? cpair{p2neg(d0.im), d0.re} : cpair{d0.im, p2neg(d0.re)};
  cpair m;
  m.re.x = __fmaf_rn(-0.5f, s.re.x, a0.re.x);
  m.re.y = __fmaf_rn(-0.5f, s.re.y, a0.re.y);
  m.im.x = __fmaf_rn(-0.5f, s.im.x, a0.im.x);
  m.im.y = __fmaf_rn(-0.5f, s.im.y, a0.im.y);
  a0 = cpadd(a0, s);
  a1.re.x = __fmaf_rn(FPM_R3, d.re.x, m.re.x);
  a1.re.y = __fmaf_rn(FPM_R3, d.re.y, m.re.y);
  a1.im.x = __fmaf_rn(FPM_R3, d.im.x, m.im.x);
  a1.im.y = __fmaf_rn(FPM_R3, d.im.y, m.im.y);
  a2.re.x = __fmaf_rn(-FPM_R3, d.re.x, m.re.x);
  a2.re.y = __fmaf_rn(-FPM_R3, d.re.y, m.re.y);
  a2.im.x = __fmaf_rn(-FPM_R3, d.im.x, m.im.x);
  a2.im.y = __fmaf_rn(-FPM_R3, d.im.y, m.im.y);
}

template <int R, int S>
struct DftP;

template <int S>
struct DftP<2, S> {
  __device__ __forceinline__ static void run(cpair *v) { dft2p<S>(v[0], v[1]); }
};

template <int S>
struct DftP<4, S> {
  __device__ __forceinline__ static void run(cpair *v) { dft4p<S>(v[0], v[1], v[2], v[3]); }
};

template <int S>
struct DftP<3, S> {
  __device__ __forceinline__ static void run(cpair *v) { dft3p<S>(v[0], v[1], v[2]); }
};

// 8 = 2 x 4, as Dft<8>
template <int S>
struct DftP<8, S> {
  __device__ __forceinline__ static void run(cpair *v) {
    cpair e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    cpair o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4p<S>(e0, e1, e2, e3);
    dft4p<S>(o0, o1, o2, o3);
    o1 = cpmul_cs<S>(o1, FPM_R2, FPM_R2);
    o3 = cpmul_cs<S>(o3, -FPM_R2, FPM_R2);
    v[0] = cpadd(e0, o0);
    v[4] = cpsub(e0, o0);
    v[1] = cpadd(e1, o1);
    v[5] = cpsub(e1, o1);
    // o2 * S i folded: e2 +/- S i o2
    if (S > 0) {
      v[2] = cpair{p2sub(e2.re, o2.im), p2add(e2.im, o2.re)};
      v[6] = cpair{p2add(e2.re, o2.im), p2sub(e2.im, o2.re)};
    } else {
      v[2] = cpair{p2add(e2.re, o2.im), p2sub(e2.im, o2.re)};
      v[6] = cpair{p2sub(e2.re, o2.im), p2add(e2.im, o2.re)};
    }
    v[3] = cpadd(e3, o3);
    v[7] = cpsub(e3, o3);
  }
};

// 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2, as Dft<16>
template <int S>
struct DftP<16, S> {
  __device__ __forceinline__ static void run(cpair *v) {
    cpair y[16];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      cpair a0 = v[n2], a1 = v[4 + n2], a2 = v[8 + n2], a3 = v[12 + n2];
      dft4p<S>(a0, a1, a2, a3);
      y[n2 * 4 + 0] = a0;
      y[n2 * 4 + 1] = a1;
      y[n2 * 4 + 2] = a2;
      y[n2 * 4 + 3] = a3;
    }
    y[1 * 4 + 1] = cpmul_cs<S>(y[5], FPM_C8, FPM_S8);
    y[1 * 4 + 2] = cpmul_cs<S>(y[6], FPM_R2, FPM_R2);
    y[1 * 4 + 3] = cpmul_cs<S>(y[7], FPM_S8, FPM_C8);
    y[2 * 4 + 1] = cpmul_cs<S>(y[9], FPM_R2, FPM_R2);
    y[2 * 4 + 2] = cpmul_si<S>(y[10]);
    y[2 * 4 + 3] = cpmul_cs<S>(y[11], -FPM_R2, FPM_R2);
    y[3 * 4 + 1] = cpmul_cs<S>(y[13], FPM_S8, FPM_C8);
    y[3 * 4 + 2] = cpmul_cs<S>(y[14], -FPM_R2, FPM_R2);
    y[3 * 4 + 3] = cpmul_cs<S>(y[15], -FPM_C8, -FPM_S8);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      cpair a0 = y[k1], a1 = y[4 + k1], a2 = y[8 + k1], a3 = y[12 + k1];
      dft4p<S>(a0, a1, a2, a3);
      v[k1] = a0;
      v[k1 + 4] = a1;
      v[k1 + 8] = a2;
      v[k1 + 12] = a3;
    }
  }
};

// 12 = 3 x 4: n = 4 n1 + n2, k = k1 + 3 k2, as Dft<12>
template <int S>
struct DftP<12, S> {
  __device__ __forceinline__ static void run(cpair *v) {
    cpair y[12];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      cpair a0 = v[n2], a1 = v[4 + n2], a2 = v[8 + n2];
      dft3p<S>(a0, a1, a2);
      y[n2 * 3 + 0] = a0;
      y[n2 * 3 + 1] = a1;
      y[n2 * 3 + 2] = a2;
    }
    y[1 * 3 + 1] = cpmul_cs<S>(y[4], FPM_R3, 0.5f);
    y[1 * 3 + 2] = cpmul_cs<S>(y[5], 0.5f, FPM_R3);
    y[2 * 3 + 1] = cpmul_cs<S>(y[7], 0.5f, FPM_R3);
    y[2 * 3 + 2] = cpmul_cs<S>(y[8], -0.5f, FPM_R3);
    y[3 * 3 + 1] = cpmul_si<S>(y[10]);
    y[3 * 3 + 2] = cpair{p2neg(y[11].re), p2neg(y[11].im)};
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
      cpair a0 = y[k1], a1 = y[3 + k1], a2 = y[6 + k1], a3 = y[9 + k1];
      dft4p<S>(a0, a1, a2, a3);
      v[k1] = a0;
      v[k1 + 3] = a1;
      v[k1 + 6] = a2;
      v[k1 + 9] = a3;
    }
  }
};

}  // namespace fpm
