// Fused per-LED update on packed FP32x2 arithmetic: every lane runs two 1-D
// transforms of the same update at once (two rows in the row phases, two
// adjacent columns in the column phase), each value pair in one FADD2 / FMUL2 /
// FFMA2 instruction (dft2.cuh).
//
// It computes exactly what run_update (update.cuh) computes, with the same
// split m = A * B, the same twiddles, the same butterflies and the same
// per-element operations in the same order, so its results are bit-identical
// to every scalar variant (up to the sign of exact zeros, which no later
// operation can turn into a different value).  What changes is the schedule:
//   phase 1  pairs of support rows: IDFT along x             -> shared "inter" [R][m]
//   phase 2  pairs of adjacent columns: IDFT along y, amplitude step, DFT along y
//   phase 3  pairs of support rows: DFT along x, spectrum and pupil updates
// A group of TPT lanes owns one pair of transforms; the exchange between the
// radix-A and radix-B passes goes through a per-group scratch of 16-byte
// chunks (re0, re1, im0, im1), one 128-bit shared-memory access per element
// pair.  "inter" holds plain interleaved complex values, swizzled in column
// pairs so that the two columns of a pair stay one aligned 16-byte chunk.
// Twiddles are read from global memory (they stay in L1) as 16-byte entries
// (w.x, w.x, w.y, w.y).
#pragma once

#include <cooperative_groups.h>
#include <cstdint>

#include "dft2.cuh"
#include "update.cuh"

namespace cg = cooperative_groups;

namespace fpm {

// Swizzled position of local column p of stored row i (box row y), row length
// w: the XOR leaves bit 0 alone, so columns 2j and 2j+1 stay adjacent and in
// order; sixteen consecutive rows of one column pair fall in eight different
// 16-byte bank groups.
__device__ __forceinline__ int inter2_swz(int y, int p) { return p ^ (((y ^ (p >> 4)) & 7) << 1); }
__device__ __forceinline__ int inter2_at(int i, int y, int p, int w) { return i * w + inter2_swz(y, p); }

template <int M_, int A_, int B_, int TPT_, int C_, int T_, int MINB_ = 1, int PF_ = 1>
struct UpdateCfg2 {
  static constexpr int M = M_, A = A_, B = B_, TPT = TPT_, C = C_, T = T_, MINB = MINB_, PF = PF_;
  static constexpr int W = M / C;          // columns of "inter" held by one CTA
  static constexpr int G = T / TPT;        // transform pairs in flight per CTA
  static constexpr int SCR = (B * (A + 1) > A * (B + 1)) ? B * (A + 1) : A * (B + 1);   // 16-byte chunks
  static constexpr int UA = (B + TPT - 1) / TPT;
  static constexpr int UB = (A + TPT - 1) / TPT;
  static constexpr int PACKED = 1;
  static_assert(A * B == M, "m = A * B");
  static_assert(A == image_split_a(M), "the tile images are laid out for the canonical split of m");
  static_assert(32 % TPT == 0 && T % 32 == 0, "groups must not straddle warps");
  static_assert(W % 16 == 0, "inter rows are swizzled in groups of 16");
  static_assert(T <= 512, "the normaliser holds one partial per warp in 16 slots");
  static_assert(W % A == 0, "a CTA's columns hold whole radix-A groups (owner and column known at compile time)");
  static_assert(UB == 1, "one radix-A unit per lane in the row phases");
  // shared memory in bytes for R support rows: [partials][inter R x W][scratch]
  static size_t smem_bytes(int rows) {
    return 64 * sizeof(float) + (size_t)rows * W * sizeof(float2) + (size_t)G * SCR * sizeof(float4);
  }
};

__device__ __forceinline__ cpair cp_from_chunk(float4 q) { return cpair{make_float2(q.x, q.y), make_float2(q.z, q.w)}; }
__device__ __forceinline__ float4 cp_to_chunk(cpair v) { return make_float4(v.re.x, v.re.y, v.im.x, v.im.y); }
// the two values of a pair as interleaved complex numbers
__device__ __forceinline__ float2 cp_first(cpair v) { return make_float2(v.re.x, v.im.x); }
__device__ __forceinline__ float2 cp_second(cpair v) { return make_float2(v.re.y, v.im.y); }
__device__ __forceinline__ cpair cp_join(float2 a, float2 b) { return cpair{make_float2(a.x, b.x), make_float2(a.y, b.y)}; }

// twiddle j of a packed table: (w.x, w.x), (w.y, w.y), (-w.y, -w.y)
struct TwP {
  float2 wx, wy, nwy;
};
__device__ __forceinline__ TwP tw2_at(const float4 *t, int j) {
  const float4 q = __ldg(t + j);
  const float2 wy = make_float2(q.z, q.w);
  return TwP{make_float2(q.x, q.y), wy, p2neg(wy)};
}
__device__ __forceinline__ cpair cpmul_tw(cpair a, TwP w) { return cpmul_w(a, w.wx, w.wy, w.nwy); }

template <class Cfg, typename Img>
__device__ __forceinline__ void run_update2(const UpdateArgs &a, int4 item, float2 *smem) {
  constexpr int M = Cfg::M, A = Cfg::A, B = Cfg::B, TPT = Cfg::TPT, C = Cfg::C, T = Cfg::T;
  constexpr int W = Cfg::W, G = Cfg::G, SCR = Cfg::SCR;
  const int rows = a.rows;
  const float4 *__restrict__ twi = a.tw2_inv;
  const float4 *__restrict__ twf = a.tw2_fwd;
  float *red = reinterpret_cast<float *>(smem);
  float2 *inter = smem + 32;              // after 64 floats of partials
  float4 *scratch_all = reinterpret_cast<float4 *>(inter + (size_t)rows * W);

  const int tid = threadIdx.x;
  const int g = tid / TPT, tl = tid % TPT;
  const unsigned lane = tid & 31;
  const unsigned gmask = (TPT == 32) ? 0xffffffffu : (((1u << TPT) - 1u) << (lane & ~(unsigned)(TPT - 1)));
  float4 *scr = scratch_all + g * SCR;

  int q = 0;
  float2 *inter_of[C];
  if constexpr (C > 1) {
    cg::cluster_group cl = cg::this_cluster();
    q = (int)cl.block_rank();
#pragma unroll
    for (int r = 0; r < C; ++r) inter_of[r] = cl.map_shared_rank(inter, r);
  } else {
    inter_of[0] = inter;
  }

  const int tile = item.x, led = item.y, slot = item.z;
  const int2 sh = a.shifts[(size_t)tile * a.n_leds + led];
  const int n = a.n;
  const int oy = n / 2 + sh.x - M / 2, ox = n / 2 + sh.y - M / 2;
  float2 *__restrict__ spec = a.spec + (size_t)tile * n * n + (size_t)oy * n + ox;   // box origin
  const size_t mm = (size_t)M * M;
  const float2 *__restrict__ pup = a.pup + (size_t)tile * mm;
  float2 *dp_out = a.dpup ? a.dpup + ((size_t)tile * a.slots + slot) * mm : nullptr;
  const Img *img = reinterpret_cast<const Img *>(a.images) + tile_image_offset(tile, led, a.n_leds, M) +
                   (size_t)q * W * M;

  // rows of the support handled by this CTA in phases 1 and 3, taken in pairs
  const int rpc = (rows + C - 1) / C;
  const int r0 = q * rpc, r1 = min(rows, r0 + rpc);
  const int npairs = (r1 - r0 + 1) / 2;
  const int2 no_chord = make_int2(1, 0);    // empty: the missing second row of an odd count

  // ---- phase 1: IDFT along x of pairs of support rows ---------------------
  float omax = 0.f, pmax = 0.f;
  for (int pr = g; pr < npairs; pr += G) {
    const int i0 = r0 + 2 * pr, i1 = i0 + 1;
    const bool has1 = i1 < r1;
    const int by0 = a.y_lo + i0, by1 = a.y_lo + i1;
    const int2 ch0 = a.chords[by0], ch1 = has1 ? a.chords[by1] : no_chord;
    const float2 *__restrict__ s0 = spec + (size_t)by0 * n;
    const float2 *__restrict__ s1 = spec + (size_t)by1 * n;
    const float2 *__restrict__ p0 = pup + (size_t)by0 * M;
    const float2 *__restrict__ p1 = pup + (size_t)by1 * M;
    // the group's next pair of rows into L2 while this one is worked on
    if (pr + G < npairs && tl * 16 < M) {
      const int nb = by0 + 2 * G;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (i0 + 2 * G + r < r1) {
          const int2 nc = a.chords[nb + r];
          if (tl * 16 + 15 >= nc.x && tl * 16 <= nc.y) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(spec + (size_t)(nb + r) * n + tl * 16));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(pup + (size_t)(nb + r) * M + tl * 16));
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < Cfg::UA; ++u) {
      const int b = tl + u * TPT;
      if (b < B) {
        cpair v[A];
#pragma unroll
        for (int aa = 0; aa < A; ++aa) {
          const int x = B * aa + b;
          const bool in0 = x >= ch0.x && x <= ch0.y, in1 = x >= ch1.x && x <= ch1.y;
          const float2 z = make_float2(0.f, 0.f);
          const cpair o = cp_join(in0 ? s0[x] : z, in1 ? s1[x] : z);
          const cpair p = cp_join(in0 ? p0[x] : z, in1 ? p1[x] : z);
          const float2 o2 = cpabs2(o), pp2 = cpabs2(p);
          omax = fmaxf(omax, fmaxf(o2.x, o2.y));
          pmax = fmaxf(pmax, fmaxf(pp2.x, pp2.y));
          v[aa] = cpmul(o, p);
        }
        DftP<A, 1>::run(v);
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1)
          scr[b * (A + 1) + k1] = cp_to_chunk(k1 == 0 ? v[0] : cpmul_tw(v[k1], tw2_at(twi, k1 * B + b)));
      }
    }
    __syncwarp(gmask);
#pragma unroll
    for (int u = 0; u < Cfg::UB; ++u) {
      const int k1 = tl + u * TPT;
      if (k1 < A) {
        cpair v[B];
#pragma unroll
        for (int bb = 0; bb < B; ++bb) v[bb] = cp_from_chunk(scr[bb * (A + 1) + k1]);
        DftP<B, 1>::run(v);
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
          // x = k1 + A k2 with k1 < A and W a multiple of A: the owning CTA and the
          // group of A columns are fixed by k2 alone
          const int owner = (A * k2) / W;
          const int p = k1 + (A * k2) % W;
          inter_of[owner][inter2_at(i0, by0, p, W)] = cp_first(v[k2]);
          if (has1) inter_of[owner][inter2_at(i1, by1, p, W)] = cp_second(v[k2]);
        }
      }
    }
    __syncwarp(gmask);
  }
  // normalisers: max |O_box_old|^2 and max |P|^2 over the support, over the whole cluster
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    omax = fmaxf(omax, __shfl_xor_sync(0xffffffffu, omax, o));
    pmax = fmaxf(pmax, __shfl_xor_sync(0xffffffffu, pmax, o));
  }
  if (lane == 0) {
    red[tid >> 5] = omax;
    red[16 + (tid >> 5)] = pmax;
  }
  if constexpr (C > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
  if (tid >= T - 32) {
    const int l = tid - (T - 32), wi = l & 15;
    float v = (wi < T / 32) ? red[l] : 0.f;            // lanes 0-15: |O|^2, 16-31: |P|^2
    if constexpr (C > 1) {
      cg::cluster_group cl = cg::this_cluster();
      for (int r = 0; r < C; ++r)
        if (r != q && wi < T / 32) v = fmaxf(v, cl.map_shared_rank(red, r)[l]);
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (l == 0) red[32] = v;
    if (l == 16) red[33] = v;
  }

  // ---- phase 2: pairs of adjacent columns: IDFT along y, amplitude, DFT along y
  const int y_lo = a.y_lo, y_hi = a.y_lo + rows - 1;
  unsigned in_mask[Cfg::UA], out_mask[Cfg::UA];
#pragma unroll
  for (int u = 0; u < Cfg::UA; ++u) {
    const int b = tl + u * TPT;
    in_mask[u] = 0;
    out_mask[u] = 0;
#pragma unroll
    for (int aa = 0; aa < A; ++aa) {
      const int y = B * aa + b;
      if (b < B && y >= y_lo && y <= y_hi) in_mask[u] |= 1u << aa;
    }
#pragma unroll
    for (int k2 = 0; k2 < A; ++k2) {
      const int y = b + B * k2;
      if (b < B && y >= y_lo && y <= y_hi) out_mask[u] |= 1u << k2;
    }
  }
  // measured pixels of this lane's rows y = k1 + A k2 in the two columns
  ImgCol<Img, B> meas[Cfg::UB][2];
  auto fetch = [&](int col, ImgCol<Img, B> (&dst)[Cfg::UB][2]) {
#pragma unroll
    for (int u = 0; u < Cfg::UB; ++u) {
      const int k1 = tl + u * TPT;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (k1 < A && col < W) dst[u][h].load(img + (size_t)(col + h) * M + k1 * B);
        else dst[u][h].zero();
      }
    }
  };
  const float2 inv_counts2 = p2dup(a.inv_counts);
  const float2 minnorm2 = p2dup(1.17549435e-38f);
  (void)minnorm2;
  if constexpr (Cfg::PF) fetch(2 * g, meas);
  for (int c = 2 * g; c < W; c += 2 * G) {
    ImgCol<Img, B> next[Cfg::PF ? Cfg::UB : 1][2];
    if constexpr (Cfg::PF) fetch(c + 2 * G, next);
    else fetch(c, meas);
#pragma unroll
    for (int u = 0; u < Cfg::UA; ++u) {
      const int b = tl + u * TPT;
      if (b < B) {
        cpair v[A];
        const float2 *col_base = inter + (b - y_lo) * W;   // row y = B aa + b is stored at i = y - y_lo
#pragma unroll
        for (int aa = 0; aa < A; ++aa) {
          if ((in_mask[u] >> aa) & 1u) {
            const float4 qv = *reinterpret_cast<const float4 *>(col_base + aa * B * W + inter2_swz(B * aa + b, c));
            v[aa] = cp_join(make_float2(qv.x, qv.y), make_float2(qv.z, qv.w));
          } else {
            v[aa] = cpzero();
          }
        }
        DftP<A, 1>::run(v);
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1)
          scr[b * (A + 1) + k1] = cp_to_chunk(k1 == 0 ? v[0] : cpmul_tw(v[k1], tw2_at(twi, k1 * B + b)));
      }
    }
    __syncwarp(gmask);
    cpair keep[Cfg::UB][B];
#pragma unroll
    for (int u = 0; u < Cfg::UB; ++u) {
      const int k1 = tl + u * TPT;
      if (k1 < A) {
        cpair *v = keep[u];
#pragma unroll
        for (int bb = 0; bb < B; ++bb) v[bb] = cp_from_chunk(scr[bb * (A + 1) + k1]);
        DftP<B, 1>::run(v);
        // amplitude step at y = k1 + A k2, as in run_update: sqrt(I)/|phi~| =
        // I / sqrt(I |phi~|^2), the argument held at FLT_MIN or above; pixels
        // with phi~ = 0 take sqrt(I)
        unsigned zmask = 0;
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
          float2 in;
          if constexpr (sizeof(Img) == 2) {
            // 16-bit counts placed in the mantissa of 2^23 (exact), then 2^23
            // subtracted and scaled, both pixels in one instruction each
            const unsigned w0 = meas[u][0].w[k2 >> 1], w1 = meas[u][1].w[k2 >> 1];
            const unsigned sel = (k2 & 1) ? 0x7632u : 0x7610u;
            const float2 bits = make_float2(__uint_as_float(__byte_perm(w0, 0x4B000000u, sel)),
                                            __uint_as_float(__byte_perm(w1, 0x4B000000u, sel)));
            in = p2mul(p2add(bits, p2dup(-8388608.0f)), inv_counts2);
          } else {
            in = make_float2(meas[u][0].intensity(k2, a.inv_counts), meas[u][1].intensity(k2, a.inv_counts));
          }
          const cpair f = v[k2];
          const float2 m2 = cpabs2(f);
          const float2 xm = p2mul(in, m2);
          const float2 r = make_float2(rsqrtf(fmaxf(xm.x, 1.17549435e-38f)), rsqrtf(fmaxf(xm.y, 1.17549435e-38f)));
          v[k2] = cpscale(f, p2mul(in, r));
          zmask |= ((m2.x > 0.f) ? 0u : (1u << k2)) | ((m2.y > 0.f) ? 0u : (1u << (k2 + 16)));
        }
        if (zmask) {
#pragma unroll
          for (int k2 = 0; k2 < B; ++k2) {
            if ((zmask >> k2) & 1u) {
              v[k2].re.x = sqrtf(meas[u][0].intensity(k2, a.inv_counts));
              v[k2].im.x = 0.f;
            }
            if ((zmask >> (k2 + 16)) & 1u) {
              v[k2].re.y = sqrtf(meas[u][1].intensity(k2, a.inv_counts));
              v[k2].im.y = 0.f;
            }
          }
        }
        DftP<B, -1>::run(v);
      }
    }
    __syncwarp(gmask);   // everyone has read scr
#pragma unroll
    for (int u = 0; u < Cfg::UB; ++u) {
      const int k1 = tl + u * TPT;
      if (k1 < A) {
#pragma unroll
        for (int kk = 0; kk < B; ++kk)
          scr[k1 * (B + 1) + kk] = cp_to_chunk(kk == 0 ? keep[u][0] : cpmul_tw(keep[u][kk], tw2_at(twf, kk * A + k1)));
      }
    }
    __syncwarp(gmask);
#pragma unroll
    for (int u = 0; u < Cfg::UA; ++u) {
      const int kk = tl + u * TPT;   // k1' in [0, B)
      if (kk < B) {
        cpair v[A];
#pragma unroll
        for (int bb = 0; bb < A; ++bb) v[bb] = cp_from_chunk(scr[bb * (B + 1) + kk]);
        DftP<A, -1>::run(v);
        float2 *col_base = inter + (kk - y_lo) * W;
#pragma unroll
        for (int k2 = 0; k2 < A; ++k2)
          if ((out_mask[u] >> k2) & 1u) {
            const float2 f0 = cp_first(v[k2]), f1 = cp_second(v[k2]);
            *reinterpret_cast<float4 *>(col_base + k2 * B * W + inter2_swz(kk + B * k2, c)) =
                make_float4(f0.x, f0.y, f1.x, f1.y);
          }
      }
    }
    __syncwarp(gmask);
#pragma unroll
    for (int u = 0; u < Cfg::UB; ++u)
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if constexpr (Cfg::PF) meas[u][h] = next[u][h];
  }
  if constexpr (C > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }

  const float onorm = red[32], pn = red[33];
  const float inv_on = (onorm > 0.f) ? 1.f / onorm : 0.f;
  const float inv_pn = 1.f / pn;
  const float2 inv_on2 = p2dup(inv_on), inv_pn2 = p2dup(inv_pn), scale2 = p2dup(a.scale);

  // ---- phase 3: DFT along x of pairs of support rows, then the updates ------
  for (int pr = g; pr < npairs; pr += G) {
    const int i0 = r0 + 2 * pr, i1 = i0 + 1;
    const bool has1 = i1 < r1;
    const int by0 = a.y_lo + i0, by1 = a.y_lo + i1;
    const int2 ch0 = a.chords[by0], ch1 = has1 ? a.chords[by1] : no_chord;
    float2 *__restrict__ s0 = spec + (size_t)by0 * n;
    float2 *__restrict__ s1 = spec + (size_t)by1 * n;
    const float2 *__restrict__ p0 = pup + (size_t)by0 * M;
    const float2 *__restrict__ p1 = pup + (size_t)by1 * M;
    // O_box_old and P of both rows at this lane's outputs x = kk + B k2, fetched
    // before the transforms so that their latency overlaps them
    cpair ov[Cfg::UA][A], pv[Cfg::UA][A];
#pragma unroll
    for (int u = 0; u < Cfg::UA; ++u) {
      const int kk = tl + u * TPT;
#pragma unroll
      for (int k2 = 0; k2 < A; ++k2) {
        const int x = kk + B * k2;
        const bool in0 = kk < B && x >= ch0.x && x <= ch0.y, in1 = kk < B && x >= ch1.x && x <= ch1.y;
        const float2 z = make_float2(0.f, 0.f);
        ov[u][k2] = cp_join(in0 ? s0[x] : z, in1 ? s1[x] : z);
        pv[u][k2] = cp_join(in0 ? p0[x] : z, in1 ? p1[x] : z);
      }
    }
#pragma unroll
    for (int u = 0; u < Cfg::UB; ++u) {
      const int b2 = tl + u * TPT;   // b' in [0, A)
      if (b2 < A) {
        cpair v[B];
#pragma unroll
        for (int aa = 0; aa < B; ++aa) {
          const int owner = (A * aa) / W;          // x = A aa + b2, b2 < A
          const int p = b2 + (A * aa) % W;
          const float2 f0 = inter_of[owner][inter2_at(i0, by0, p, W)];
          const float2 f1 = has1 ? inter_of[owner][inter2_at(i1, by1, p, W)] : make_float2(0.f, 0.f);
          v[aa] = cp_join(f0, f1);
        }
        DftP<B, -1>::run(v);
#pragma unroll
        for (int kk = 0; kk < B; ++kk)
          scr[b2 * (B + 1) + kk] = cp_to_chunk(kk == 0 ? v[0] : cpmul_tw(v[kk], tw2_at(twf, kk * A + b2)));
      }
    }
    __syncwarp(gmask);
#pragma unroll
    for (int u = 0; u < Cfg::UA; ++u) {
      const int kk = tl + u * TPT;
      if (kk < B) {
        cpair v[A];
#pragma unroll
        for (int bb = 0; bb < A; ++bb) v[bb] = cp_from_chunk(scr[bb * (B + 1) + kk]);
        DftP<A, -1>::run(v);
#pragma unroll
        for (int k2 = 0; k2 < A; ++k2) {
          const int x = kk + B * k2;
          const bool in0 = x >= ch0.x && x <= ch0.y, in1 = x >= ch1.x && x <= ch1.y;
          if (in0 || in1) {
            const cpair o = ov[u][k2], p = pv[u][k2];
            const cpair phi = cpmul(o, p);
            const cpair d = cpsub(cpscale(v[k2], scale2), phi);
            const cpair pc = cpmulc(d, p);        // D * conj(P)
            const cpair nw = cpair{p2fma(pc.re, inv_pn2, o.re), p2fma(pc.im, inv_pn2, o.im)};
            if (in0) s0[x] = cp_first(nw);
            if (in1) s1[x] = cp_second(nw);
            if (dp_out) {
              const cpair dpv = cpscale(cpmulc(d, o), inv_on2);   // D * conj(O_old)
              if (in0) dp_out[(size_t)by0 * M + x] = cp_first(dpv);
              if (in1) dp_out[(size_t)by1 * M + x] = cp_second(dpv);
            }
          }
        }
      }
    }
    __syncwarp(gmask);
  }
  // keep this CTA's shared memory alive until the cluster is done reading it
  if constexpr (C > 1) {
    cg::this_cluster().sync();
  }
}

template <class Cfg, typename Img>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB) update2_kernel(const __grid_constant__ UpdateArgs a, long long item0) {
  extern __shared__ float4 smem_raw[];
  const int4 item = a.items[item0 + blockIdx.x / Cfg::C];
  run_update2<Cfg, Img>(a, item, reinterpret_cast<float2 *>(smem_raw));
}

}  // namespace fpm
