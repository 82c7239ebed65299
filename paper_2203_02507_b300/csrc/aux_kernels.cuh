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
  const float2 *src;           // input lines at the same offsets, or null (in place)
  const float2 *tw;            // [len] exp(sign 2 pi i j / len)
  long long batch_stride;      // elements between batches
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
};

// Shared-memory position of line sample i: one pad slot per 16 samples, so a
// butterfly's R outputs written with unit stride by consecutive threads (the
// first Stockham pass) fall in different banks.
__device__ __forceinline__ int line_pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int line_padded_len(int len) { return len + len / 16 + 1; }

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
  const long long off = (line0 / f.lines_per_batch) * f.batch_stride + (line0 % f.lines_per_batch) * f.line_stride;
  const int l0 = (int)(line0 % f.lines_per_batch);
  const int plen = line_padded_len(len);
  float2 *base = f.data + off;
  const float2 *in = (f.src ? f.src : f.data) + off;
  // sample e of line c at e * elem_stride + c (adjacent lines: line_stride 1)
  for (int i = threadIdx.x; i < len * lpc; i += blockDim.x) {
    const int e = i / lpc, c = i - e * lpc;
    line_buf[(size_t)c * 2 * plen + line_pad(e)] = in[(long long)e * f.elem_stride + c];
  }
  __syncthreads();
  // the CTA's threads form lpc groups, one per line; passes run in lockstep
  const int nt = blockDim.x / lpc, grp = threadIdx.x / nt, t = threadIdx.x - grp * nt;
  float2 *b0 = line_buf + (size_t)grp * 2 * plen;
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
  for (int i = threadIdx.x; i < len * lpc; i += blockDim.x) {
    const int e = i / lpc, c = i - e * lpc;
    float2 v = line_buf[(size_t)c * 2 * plen + cur * plen + line_pad(e)];
    if (f.finish != 0.f) {
      const float sc = ((e + l0 + c) & 1) ? -f.finish : f.finish;
      v = make_float2(__fmul_rn(v.x, sc), __fmul_rn(v.y, sc));
    }
    base[(long long)e * f.elem_stride + c] = v;
  }
}

// Lines of 256 (16 x 16) or 1024 (16 x 16 x 4) samples with the butterflies in
// registers: the same Stockham passes, twiddles and radix order as
// fft_lines_kernel (so the same results bit for bit), with compile-time
// indices, the first pass fed straight from global memory and the last pass
// stored straight to it where the lines are contiguous (elem_stride 1).  Lines
// whose samples are strided (line_stride 1, elem_stride > 1) are staged through
// shared memory G adjacent lines at a time, so every 32-byte sector is used
// whole.  G lines per CTA, LEN / 16 threads per line; shared memory G *
// line_padded_len(LEN) float2 (one buffer, a barrier between the reads and the
// writes of each pass).
template <int S, int LEN, int G>
__global__ void __launch_bounds__(G *(LEN / 16), G *(LEN / 16) >= 512 ? 2 : 3)
    fft_lines_reg_kernel(const __grid_constant__ FftLines f) {
  static_assert(LEN == 256 || LEN == 1024, "lengths 16 x 16 and 16 x 16 x 4");
  constexpr int NT = LEN / 16;                 // threads per line
  constexpr int PL = line_padded_len(LEN);
  extern __shared__ float2 line_buf[];
  const int g = threadIdx.x / NT, t = threadIdx.x - g * NT;
  const long long line0 = (long long)blockIdx.x * G;
  const bool rows = f.elem_stride == 1;
  // rows: each group's own line; strided: G adjacent lines of one batch
  const long long line = rows ? line0 + g : line0;
  const long long off = (line / f.lines_per_batch) * f.batch_stride + (line % f.lines_per_batch) * f.line_stride;
  const int lb = (int)(line % f.lines_per_batch);     // index of the (first) line within its batch
  const float2 *in = (f.src ? f.src : f.data) + off;
  float2 *out = f.data + off;
  float2 *xs = line_buf + (size_t)g * PL;
  float2 v[16];
  if (rows) {
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = in[t + r * NT];
  } else {
    // 16 loads a thread, all in flight before their shared-memory stores
    float2 u[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int i = threadIdx.x + q * G * NT, e = i / G, c = i - e * G;
      u[q] = in[(long long)e * f.elem_stride + c];
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
    if (r > 0 && k2 > 0) v[r] = cmul(v[r], f.tw[k2 * r * step2]);
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
        if (r > 0 && j > 0) w[q][r] = cmul(w[q][r], f.tw[j * r]);
      }
      Dft<4, S>::run(w[q]);
    }
    if (rows) {
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
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int i = threadIdx.x + q * G * NT, e = i / G, c = i - e * G;
    out[(long long)e * f.elem_stride + c] = finish(line_buf[(size_t)c * PL + line_pad(e)], e, c);
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
// corrections of each in flight together, no table read first.  Rows are cut
// into `parts` chunks; merge_rows does chunk `part` with the threads
// [t0, t0 + nt) of the calling CTA(s) (t0 and nt multiples of 32).
constexpr int kMergeSlots = 8;   // corrections loaded together
constexpr int kMergePairs = 2;   // pixel pairs per lane in flight

__device__ __forceinline__ void merge_rows(float2 *__restrict__ pup, const float2 *__restrict__ dpup, int t, int ns,
                                           int part, int parts, int y_lo, int rows, int m, int slots, int disc,
                                           int t0, int nt) {
  if (ns <= 0) return;
  const int rpp = (rows + parts - 1) / parts;
  const int r0 = part * rpp, r1 = min(rows, r0 + rpp);
  const int hp = m / 2;                                   // pixel pairs per row
  const size_t mm2 = (size_t)m * m / 2;                   // float4 per pupil
  float4 *p = reinterpret_cast<float4 *>(pup + (size_t)t * m * m);
  const float4 *d = reinterpret_cast<const float4 *>(dpup + (size_t)t * slots * m * m);
  const int lane = t0 & 31, warp = t0 >> 5, warps = nt >> 5;
  for (int r = r0 + warp; r < r1; r += warps) {
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
