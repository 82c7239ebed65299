// Kernels off the per-LED inner loop: a general batched 1-D FFT (Stockham
// autosort, radix 2/3/4, one line per CTA in shared memory) used by the initial
// guess and the forward-model simulator, the initial-guess gather/place steps,
// the pupil-correction merge with the max|P|^2 normaliser, and the simulator's
// crop and intensity steps.
#pragma once

#include <cstdint>

#include "dft.cuh"
#include "tile_images.cuh"
#include "update_args.h"

namespace fpm {

constexpr int kMaxFftLen = 2048;
constexpr int kMaxRadices = 12;

struct FftLines {
  float2 *data;                // output lines (and input, unless src is set)
  const float2 *src;           // input lines at the same offsets within a batch, or null (in place)
  const float2 *tw;            // [len] exp(sign 2 pi i j / len)
  // optional, lengths 256 and 1024: the same twiddles in the order the register
  // kernel's passes read them, so that a warp's loads share cache lines:
  // [(r - 1) 16 + k] = tw[k r len / 256] (r < 16, k < 16), then for length 1024
  // [240 + (r - 1) 256 + j] = tw[j r] (r < 4, j < 256)
  const float2 *tw_pass;
  long long batch_stride;      // elements between batches
  long long src_batch_stride;  // elements between batches of src (the launcher sets batch_stride when 0)
  long long line_stride;       // elements between lines of a batch
  long long elem_stride;       // elements between samples of a line
  int lines_per_batch;
  int len;
  int nrad;
  int radix[kMaxRadices];
  int lines_per_cta;           // 1, or that many adjacent lines (line_stride 1), moved
                               // together so each 32-byte sector is used whole
  float finish;                // 0, or: output (e, l) times finish * (-1)^(e + l),
                               // e the sample and l the line index within its batch
  // Field-of-view output (strided lines only, one batch = one tile): with fov set,
  // output sample e of line l of batch b is not stored in `data` but, where it
  // lies in the rows and columns tile t = fov_tile0 + b keeps, multiplied by
  // fov_weight[t] into the stitched image at (i (N - ov) + e, j (N - ov) + l),
  // (i, j) = the tile's grid position, N = len.
  float2 *fov;
  const float2 *fov_weight;
  long long fov_w;             // row length of the stitched image
  int fov_ov, fov_tiles_y, fov_tiles_x, fov_tile0;
  int fov_tile_step;           // tile index step from one batch to the next (the launcher sets 1 when 0)
  // Band sums of contiguous lines (elem_stride 1): with band set, line l of the
  // launch also writes band[3 l + 0] = sum_{e < band_ov} (-1)^e y_e,
  // band[3 l + 1] = sum_{e >= len - band_ov} (-1)^e y_e (y the output before
  // any finish) and band[3 l + 2] = its input sample len / 2.
  float2 *band;
  int band_ov;
};

// Rows [r0, r1) that tile row i (of k_tiles, N = n, shared band ov) keeps in the
// stitched image (Eq. 1 read as: a neighbour pair's first image up to r - ov/2).
__host__ __device__ inline void stitch_kept(int i, int k_tiles, int n, int ov, int *r0, int *r1) {
  *r0 = i > 0 ? ov - ov / 2 : 0;
  *r1 = i < k_tiles - 1 ? n - ov / 2 : n;
}

// Where the lines a CTA stores go: every line of a CTA lies in one batch, so
// with a field-of-view output the tile, its grid position, the rows and the
// columns it keeps are fixed per CTA (computed once by line_target).
struct LineTarget {
  float2 *dst;                 // sample e of line l0 + c lands at dst[e * es + c]
  long long es;
  int y0, y1, x0, x1;          // kept samples e in [y0, y1), lines l0 + c in [x0, x1)
  int l0;
  float2 w;                    // tile weight
};
__device__ __forceinline__ LineTarget line_target(const FftLines &f, float2 *base, long long line_first) {
  LineTarget lt;
  if (!f.fov) {
    lt.dst = base;
    lt.es = f.elem_stride;
    lt.y0 = 0;
    lt.y1 = 1 << 30;
    lt.x0 = 0;
    lt.x1 = 1 << 30;
    lt.l0 = 0;
    lt.w = make_float2(1.f, 0.f);
    return lt;
  }
  const int b = (int)(line_first / f.lines_per_batch);
  const int x = (int)(line_first - (long long)b * f.lines_per_batch);
  const int t = f.fov_tile0 + b * f.fov_tile_step, i = t / f.fov_tiles_x, j = t - i * f.fov_tiles_x;
  const int stride = f.len - f.fov_ov;
  stitch_kept(i, f.fov_tiles_y, f.len, f.fov_ov, &lt.y0, &lt.y1);
  stitch_kept(j, f.fov_tiles_x, f.len, f.fov_ov, &lt.x0, &lt.x1);
  lt.l0 = x;
  lt.dst = f.fov + (long long)i * stride * f.fov_w + (long long)j * stride + x;
  lt.es = f.fov_w;
  lt.w = f.fov_weight[t];
  return lt;
}
// Store of finished output sample e of the CTA's line c.
__device__ __forceinline__ void line_store(const FftLines &f, const LineTarget &lt, int e, int c, float2 v) {
  if (!f.fov) {
    lt.dst[(long long)e * lt.es + c] = v;
    return;
  }
  if (e < lt.y0 || e >= lt.y1 || lt.l0 + c < lt.x0 || lt.l0 + c >= lt.x1) return;
  __stcs(lt.dst + (long long)e * lt.es + c, cmul(lt.w, v));   // written once: evict first
}

// Band sums of one line from its outputs: (-1)^e y_e over e < ov and over
// e >= len - ov, accumulated into *lo / *hi.
__device__ __forceinline__ void band_add(float2 y, int e, int len, int ov, float2 *lo, float2 *hi) {
  if (e >= ov && e < len - ov) return;
  const float2 v = (e & 1) ? make_float2(-y.x, -y.y) : y;
  if (e < ov) *lo = make_float2(__fadd_rn(lo->x, v.x), __fadd_rn(lo->y, v.y));
  else *hi = make_float2(__fadd_rn(hi->x, v.x), __fadd_rn(hi->y, v.y));
}
// Sum over the `width` consecutive lanes of a warp (width a power of 2 <= 32), fixed order.
template <int W>
__device__ __forceinline__ float2 lanes_sum(float2 a) {
#pragma unroll
  for (int s = W / 2; s > 0; s >>= 1) {
    a.x = __fadd_rn(a.x, __shfl_xor_sync(0xffffffffu, a.x, s));
    a.y = __fadd_rn(a.y, __shfl_xor_sync(0xffffffffu, a.y, s));
  }
  return a;
}

// Shared-memory position of line sample i: one pad slot per 16 samples, so a
// butterfly's R outputs written with unit stride by consecutive threads (the
// first Stockham pass) fall in different banks.
__device__ __forceinline__ int line_pad(int i) { return i + (i >> 4); }
// Spacing of lines in shared memory: a half-warp moving a strided tile touches
// g adjacent lines at 16 / g samples each, which fall in distinct bank pairs when
// the spacing is odd for g = 16 and 2 mod 16 for g = 8 (and for 4 lines at twice
// the spacing).
__host__ __device__ constexpr int line_padded_len(int len, int g = 8) { return len + len / 16 + (g == 16 ? 1 : 2); }

// Stockham pass: R-point butterflies on strided inputs, autosorted outputs,
// butterflies j = t, t + nt, ... done by threads t of a group of nt.
template <int R, int S>
__device__ __forceinline__ void stockham_pass(const float2 *x, float2 *y, const float2 *tw, int len, int ns, int t,
                                              int nt) {
  const int span = len / R;
  for (int j = t; j < span; j += nt) {
    const int k = j % ns;
    const int step = len / (ns * R);
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      v[r] = x[line_pad(j + r * span)];
      if (r > 0 && k > 0) v[r] = cmul(v[r], tw[k * r * step]);
    }
    Dft<R, S>::run(v);
    const int base = (j / ns) * ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) y[line_pad(base + r * ns)] = v[r];
  }
}

// lines_per_cta lines per CTA; unnormalised DFT with exp(S 2 pi i n k / len).
// Dynamic shared memory: lines_per_cta * 2 * line_padded_len(len) float2.
template <int S, int LPC>
__global__ void fft_lines_kernel(const __grid_constant__ FftLines f) {
  extern __shared__ float2 line_buf[];
  constexpr int lpc = LPC;
  const int len = f.len;
  const long long line0 = (long long)blockIdx.x * lpc;
  const long long b0i = line0 / f.lines_per_batch, loff = (line0 % f.lines_per_batch) * f.line_stride;
  const long long off = b0i * f.batch_stride + loff;
  const int l0 = (int)(line0 % f.lines_per_batch);
  const int plen = line_padded_len(len);
  float2 *base = f.data + off;
  const float2 *in = f.src ? f.src + b0i * f.src_batch_stride + loff : f.data + off;
  // sample e of line c at e * elem_stride + c (adjacent lines: line_stride 1)
  for (int i = threadIdx.x; i < len * lpc; i += blockDim.x) {
    const int e = i / lpc, c = i - e * lpc;
    line_buf[(size_t)c * 2 * plen + line_pad(e)] = in[(long long)e * f.elem_stride + c];
  }
  __syncthreads();
  // the CTA's threads form lpc groups, one per line; passes run in lockstep
  const int nt = blockDim.x / lpc, grp = threadIdx.x / nt, t = threadIdx.x - grp * nt;
  float2 *b0 = line_buf + (size_t)grp * 2 * plen;
  const float2 mid = b0[line_pad(len / 2)];           // the input sample len / 2 (band sums)
  int cur = 0, ns = 1;
  for (int p = 0; p < f.nrad; ++p) {
    const int r = f.radix[p];
    float2 *x = b0 + cur * plen, *y = b0 + (cur ^ 1) * plen;
    if (r == 16) stockham_pass<16, S>(x, y, f.tw, len, ns, t, nt);
    else if (r == 8) stockham_pass<8, S>(x, y, f.tw, len, ns, t, nt);
    else if (r == 4) stockham_pass<4, S>(x, y, f.tw, len, ns, t, nt);
    else if (r == 2) stockham_pass<2, S>(x, y, f.tw, len, ns, t, nt);
    else stockham_pass<3, S>(x, y, f.tw, len, ns, t, nt);
    ns *= r;
    cur ^= 1;
    __syncthreads();
  }
  if (f.band && t < 32) {
    // the first warp of each line's group: band sums in a fixed order
    float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
    const float2 *yl = b0 + cur * plen;
    for (int e = t; e < f.band_ov; e += 32) band_add(yl[line_pad(e)], e, len, f.band_ov, &lo, &hi);
    for (int e = len - f.band_ov + t; e < len; e += 32)
      if (e >= f.band_ov) band_add(yl[line_pad(e)], e, len, f.band_ov, &lo, &hi);
    lo = lanes_sum<32>(lo);
    hi = lanes_sum<32>(hi);
    if (t == 0) {
      float2 *bo = f.band + 3 * (line0 + grp);
      bo[0] = lo;
      bo[1] = hi;
      bo[2] = mid;
    }
  }
  const LineTarget lt = line_target(f, base, line0);
  for (int i = threadIdx.x; i < len * lpc; i += blockDim.x) {
    const int e = i / lpc, c = i - e * lpc;
    float2 v = line_buf[(size_t)c * 2 * plen + cur * plen + line_pad(e)];
    if (f.finish != 0.f) {
      const float sc = ((e + l0 + c) & 1) ? -f.finish : f.finish;
      v = make_float2(__fmul_rn(v.x, sc), __fmul_rn(v.y, sc));
    }
    line_store(f, lt, e, c, v);
  }
}

// Lines of 256 (16 x 16) or 1024 (16 x 16 x 4) samples with the butterflies in
// registers: the same Stockham passes, twiddles and radix order as
// fft_lines_kernel (so the same results bit for bit), with compile-time
// indices, the first pass fed straight from global memory and the last pass
// stored straight to it where the lines are contiguous (elem_stride 1).  Lines
// whose samples are strided (line_stride 1, elem_stride > 1) are staged through
// shared memory G adjacent lines at a time, so every 32-byte sector is used
// whole.  G lines per CTA, LEN / 16 threads per line; TP: twiddles from
// f.tw_pass; shared memory G * line_padded_len(LEN, G) float2 (one buffer, a barrier between the reads and the
// writes of each pass).
template <int S, int LEN, int G, bool TP>
__global__ void __launch_bounds__(G *(LEN / 16), G *(LEN / 16) >= 512 ? 2 : 4)
    fft_lines_reg_kernel(const __grid_constant__ FftLines f) {
  static_assert(LEN == 256 || LEN == 1024, "lengths 16 x 16 and 16 x 16 x 4");
  constexpr int NT = LEN / 16;                 // threads per line
  constexpr int PL = line_padded_len(LEN, G);
  extern __shared__ float2 line_buf[];
  const int g = threadIdx.x / NT, t = threadIdx.x - g * NT;
  const long long line0 = (long long)blockIdx.x * G;
  // (1024-sample lines in groups of 8 are always strided: the launcher takes 4 for rows)
  const bool rows = (LEN != 1024 || G != 8) && f.elem_stride == 1;
  // rows: each group's own line; strided: G adjacent lines of one batch
  const long long line = rows ? line0 + g : line0;
  const long long bi = line / f.lines_per_batch, loff = (line % f.lines_per_batch) * f.line_stride;
  const long long off = bi * f.batch_stride + loff;
  const int lb = (int)(line % f.lines_per_batch);     // index of the (first) line within its batch
  const float2 *in = f.src ? f.src + bi * f.src_batch_stride + loff : f.data + off;
  float2 *out = f.data + off;
  float2 *xs = line_buf + (size_t)g * PL;
  __shared__ float2 band_red[G][(NT + 31) / 32][2];
  // band sums of contiguous lines: partial sums of each thread, then of the line
  auto band_out = [&](float2 lo, float2 hi, float2 mid) {
    constexpr int W = NT < 32 ? NT : 32;
    lo = lanes_sum<W>(lo);
    hi = lanes_sum<W>(hi);
    if constexpr (NT > 32) {
      if ((t & 31) == 0) {
        band_red[g][t >> 5][0] = lo;
        band_red[g][t >> 5][1] = hi;
      }
      __syncthreads();
      if (t == 0)
        for (int w = 1; w < NT / 32; ++w) {
          lo = cadd(lo, band_red[g][w][0]);
          hi = cadd(hi, band_red[g][w][1]);
        }
    }
    if (t == 0) {
      float2 *bo = f.band + 3 * line;
      bo[0] = lo;
      bo[1] = hi;
      bo[2] = mid;
    }
  };
  float2 v[16];
  float2 mid = make_float2(0.f, 0.f);
  if (rows) {
    // spectra are read once: evict first
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = __ldcs(in + t + r * NT);
    mid = v[8];                                   // sample LEN / 2 = 8 NT (thread 0)
  } else {
    // 16 loads a thread, all in flight before their shared-memory stores
    float2 u[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int i = threadIdx.x + q * G * NT, e = i / G, c = i - e * G;
      u[q] = __ldcs(in + (long long)e * f.elem_stride + c);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int i = threadIdx.x + q * G * NT, e = i / G, c = i - e * G;
      line_buf[(size_t)c * PL + line_pad(e)] = u[q];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = xs[line_pad(t + r * NT)];
    __syncthreads();
  }
  // pass 1: radix 16, ns = 1 (no twiddles); butterfly t, outputs 16 t + r
  Dft<16, S>::run(v);
#pragma unroll
  for (int r = 0; r < 16; ++r) xs[line_pad(16 * t + r)] = v[r];
  __syncthreads();
  // pass 2: radix 16, ns = 16; butterfly t, inputs t + r NT, outputs (t / 16) 256 + t % 16 + 16 r
  const int k2 = t % 16;
  constexpr int step2 = LEN / 256;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    v[r] = xs[line_pad(t + r * NT)];
    if (r > 0 && k2 > 0) v[r] = cmul(v[r], TP ? f.tw_pass[(r - 1) * 16 + k2] : f.tw[k2 * r * step2]);
  }
  Dft<16, S>::run(v);
  const int base2 = (t / 16) * 256 + k2;
  // the finishing sign and scale of output sample e of line lb + c
  auto finish = [&](float2 a, int e, int c) {
    if (f.finish == 0.f) return a;
    const float sc = ((e + lb + c) & 1) ? -f.finish : f.finish;
    return make_float2(__fmul_rn(a.x, sc), __fmul_rn(a.y, sc));
  };
  if constexpr (LEN == 256) {
    if (rows) {
      if (f.band) {
        float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < 16; ++r) band_add(v[r], base2 + 16 * r, LEN, f.band_ov, &lo, &hi);
        band_out(lo, hi, mid);
      }
#pragma unroll
      for (int r = 0; r < 16; ++r) out[base2 + 16 * r] = finish(v[r], base2 + 16 * r, 0);
      return;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 16; ++r) xs[line_pad(base2 + 16 * r)] = v[r];
  } else {
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 16; ++r) xs[line_pad(base2 + 16 * r)] = v[r];
    __syncthreads();
    // pass 3: radix 4, ns = 256; butterflies j = t + NT q, inputs j + 256 r, outputs j + 256 r
    float2 w[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = t + NT * q;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        w[q][r] = xs[line_pad(j + 256 * r)];
        if (r > 0 && j > 0) w[q][r] = cmul(w[q][r], TP ? f.tw_pass[240 + (r - 1) * 256 + j] : f.tw[j * r]);
      }
      Dft<4, S>::run(w[q]);
    }
    if (rows) {
      if (f.band) {
        float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int r = 0; r < 4; ++r) band_add(w[q][r], t + NT * q + 256 * r, LEN, f.band_ov, &lo, &hi);
        band_out(lo, hi, mid);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int e = t + NT * q + 256 * r;
          out[e] = finish(w[q][r], e, 0);
        }
      return;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) xs[line_pad(t + NT * q + 256 * r)] = w[q][r];
  }
  // strided lines: the G lines leave through shared memory, adjacent lines together
  __syncthreads();
  const LineTarget lt = line_target(f, out, line);
  if (f.fov) {
    // a thread stores samples e0 + q NT of line c: one column, one sign parity
    // (NT is even), so the kept-column test and weight x finish x sign are per thread
    const int c = threadIdx.x % G, e0 = threadIdx.x / G;
    if (lt.l0 + c < lt.x0 || lt.l0 + c >= lt.x1) return;
    float2 wt = lt.w;
    if (f.finish != 0.f) {
      const float sc = ((e0 + lb + c) & 1) ? -f.finish : f.finish;
      wt = make_float2(__fmul_rn(wt.x, sc), __fmul_rn(wt.y, sc));
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = e0 + q * NT;
      if (e >= lt.y0 && e < lt.y1) __stcs(lt.dst + (long long)e * lt.es + c, cmul(wt, line_buf[(size_t)c * PL + line_pad(e)]));
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int i = threadIdx.x + q * G * NT, e = i / G, c = i - e * G;
    line_store(f, lt, e, c, finish(line_buf[(size_t)c * PL + line_pad(e)], e, c));
  }
}

// sqrt of each tile's image of the first LED, as a complex m x m array per tile.
template <typename Img>
__global__ void init_gather_kernel(float2 *out, const Img *stack, long long stride_led, long long stride_row,
                                   const int2 *origins, int led, int m, int n_tiles, float inv_counts) {
  const long long total = (long long)n_tiles * m * m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i / ((long long)m * m));
    const int y = (int)((i / m) % m), x = (int)(i % m);
    const int2 o = origins[t];
    const long long off = (long long)led * stride_led + (long long)(o.x + y) * stride_row + o.y + x;
    float v;
    if constexpr (sizeof(Img) == 2) v = (float)reinterpret_cast<const unsigned short *>(stack)[off];
    else v = reinterpret_cast<const float *>(stack)[off];
    out[i] = make_float2(sqrtf(fmaxf(__fmul_rn(v, inv_counts), 0.f)), 0.f);
  }
}

// spec[t][N/2 + ky][N/2 + kx] = scale * X[t][ky mod m][kx mod m], ky, kx in [-m/2, m/2)
static __global__ void init_place_kernel(float2 *spec, const float2 *x, int m, int n, int n_tiles, float scale) {
  const long long total = (long long)n_tiles * m * m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i / ((long long)m * m));
    const int by = (int)((i / m) % m), bx = (int)(i % m);
    const int qy = (by + m / 2) % m, qx = (bx + m / 2) % m;    // DFT index of centred k = b - m/2
    const float2 v = x[(size_t)t * m * m + (size_t)qy * m + qx];
    spec[(size_t)t * n * n + (size_t)(n / 2 - m / 2 + by) * n + (n / 2 - m / 2 + bx)] = cscale(v, scale);
  }
}

// Close a wave of a tile: add its ns pupil corrections to the pupil in slot
// (= sequence) order.  Corrections are zero off the support (the update writes
// them only there and they start zeroed) and so is the pupil, so any pixel set
// that covers the support gives the same sums: each warp takes whole rows and
// its lanes the aligned pixel pairs within the row's disc bound (disc = 1; else
// the whole row), summed with 16-byte loads, two pairs and up to kMergeSlots
// corrections of each in flight together, no table read first.  Rows are dealt
// to `parts` callers in turn (row r to part r mod parts, so that every part gets
// wide rows of the disc's middle and narrow ones of its ends alike); merge_rows
// does part `part` with the threads [t0, t0 + nt) of the calling CTA(s) (t0 and
// nt multiples of 32).
constexpr int kMergeSlots = 8;   // corrections loaded together
constexpr int kMergePairs = 2;   // pixel pairs per lane in flight

__device__ __forceinline__ void merge_rows(float2 *__restrict__ pup, const float2 *__restrict__ dpup, int t, int ns,
                                           int part, int parts, int y_lo, int rows, int m, int slots, int disc,
                                           int t0, int nt) {
  if (ns <= 0) return;
  const int hp = m / 2;                                   // pixel pairs per row
  const size_t mm2 = (size_t)m * m / 2;                   // float4 per pupil
  float4 *p = reinterpret_cast<float4 *>(pup + (size_t)t * m * m);
  const float4 *d = reinterpret_cast<const float4 *>(dpup + (size_t)t * slots * m * m);
  const int lane = t0 & 31, warp = t0 >> 5, warps = nt >> 5;
  for (int r = part + parts * warp; r < rows; r += parts * warps) {
    const int by = y_lo + r;
    const int hw = disc ? disc_half_width(by, y_lo, rows) : m;
    const int plo = max(0, m / 2 - hw) >> 1, phi = min(m - 1, m / 2 + hw) >> 1;   // pairs touching the bound
    for (int pr0 = plo + lane; pr0 <= phi; pr0 += 32 * kMergePairs) {
      size_t off[kMergePairs];
      bool act[kMergePairs];
      float4 v[kMergePairs];
#pragma unroll
      for (int u = 0; u < kMergePairs; ++u) {
        const int pr = pr0 + 32 * u;
        act[u] = pr <= phi;
        off[u] = (size_t)by * hp + pr;
        v[u] = act[u] ? p[off[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      for (int s0 = 0; s0 < ns; s0 += kMergeSlots) {
        float4 a[kMergePairs][kMergeSlots];
#pragma unroll
        for (int u = 0; u < kMergePairs; ++u)
#pragma unroll
          for (int k = 0; k < kMergeSlots; ++k)
            a[u][k] = (act[u] && s0 + k < ns) ? d[(size_t)(s0 + k) * mm2 + off[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < kMergePairs; ++u)
#pragma unroll
          for (int k = 0; k < kMergeSlots; ++k)
            if (s0 + k < ns)
              v[u] = make_float4(v[u].x + a[u][k].x, v[u].y + a[u][k].y, v[u].z + a[u][k].z, v[u].w + a[u][k].w);
      }
#pragma unroll
      for (int u = 0; u < kMergePairs; ++u)
        if (act[u]) p[off[u]] = v[u];
    }
  }
}

// Grid: (entries (tile, slots), kNormParts row chunks).
static __global__ void __launch_bounds__(256) merge_kernel(float2 *__restrict__ pup, const float2 *__restrict__ dpup,
                                                           const int2 *__restrict__ entries, int y_lo, int rows, int m,
                                                           int slots, int disc) {
  const int2 e = entries[blockIdx.x];
  merge_rows(pup, dpup, e.x, e.y, blockIdx.y, kNormParts, y_lo, rows, m, slots, disc, threadIdx.x, blockDim.x);
}

// Simulator: box of the unshifted DFT spectrum times the pupil, placed in
// IDFT input order (the box's centred index b - m/2 taken modulo m).
static __global__ void sim_crop_kernel(float2 *box, const float2 *spec_dft, const float2 *pup, const int2 *shifts,
                                int led, int n_leds, int m, int n, int n_tiles) {
  const long long total = (long long)n_tiles * m * m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i / ((long long)m * m));
    const int by = (int)((i / m) % m), bx = (int)(i % m);
    const int2 s = shifts[(size_t)t * n_leds + led];
    const int ky = ((s.x + by - m / 2) % n + n) % n, kx = ((s.y + bx - m / 2) % n + n) % n;
    const float2 v = cmul(spec_dft[(size_t)t * n * n + (size_t)ky * n + kx], pup[(size_t)t * m * m + (size_t)by * m + bx]);
    const int qy = (by + m / 2) % m, qx = (bx + m / 2) % m;
    box[(size_t)t * m * m + (size_t)qy * m + qx] = v;
  }
}

static __global__ void sim_abs_kernel(float *out, const float2 *box, int led, int n_leds, int m, int n_tiles, float inv_n2) {
  const long long total = (long long)n_tiles * m * m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i / ((long long)m * m));
    const long long px = i % ((long long)m * m);
    const float2 v = cscale(box[i], inv_n2);
    out[((size_t)t * n_leds + led) * m * m + px] = cabs2(v);
  }
}

}  // namespace fpm
