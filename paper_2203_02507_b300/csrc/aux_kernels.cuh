// Kernels off the per-LED inner loop: a general batched 1-D FFT (Stockham
// autosort, radix 2/3/4, one line per CTA in shared memory) used by the initial
// guess and the forward-model simulator, the initial-guess gather/place steps,
// the pupil-correction merge with the max|P|^2 normaliser, and the simulator's
// crop and intensity steps.
#pragma once

#include <cstdint>

#include "dft.cuh"
#include "update_args.h"

namespace fpm {

constexpr int kMaxFftLen = 2048;
constexpr int kMaxRadices = 12;

struct FftLines {
  float2 *data;
  const float2 *tw;            // [len] exp(sign 2 pi i j / len)
  long long batch_stride;      // elements between batches
  long long line_stride;       // elements between lines of a batch
  long long elem_stride;       // elements between samples of a line
  int lines_per_batch;
  int len;
  int nrad;
  int radix[kMaxRadices];
};

// Stockham pass: R-point butterflies on strided inputs, autosorted outputs.
template <int R, int S>
__device__ __forceinline__ void stockham_pass(const float2 *x, float2 *y, const float2 *tw, int len, int ns) {
  const int span = len / R;
  for (int j = threadIdx.x; j < span; j += blockDim.x) {
    const int k = j % ns;
    const int step = len / (ns * R);
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      v[r] = x[j + r * span];
      if (r > 0 && k > 0) v[r] = cmul(v[r], tw[k * r * step]);
    }
    Dft<R, S>::run(v);
    const int base = (j / ns) * ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) y[base + r * ns] = v[r];
  }
}

// One CTA per line; unnormalised DFT with exp(S 2 pi i n k / len).
template <int S>
__global__ void fft_lines_kernel(const __grid_constant__ FftLines f) {
  __shared__ float2 buf[2][kMaxFftLen];
  const long long line = blockIdx.x;
  float2 *base = f.data + (line / f.lines_per_batch) * f.batch_stride +
                 (line % f.lines_per_batch) * f.line_stride;
  for (int i = threadIdx.x; i < f.len; i += blockDim.x) buf[0][i] = base[(long long)i * f.elem_stride];
  __syncthreads();
  int cur = 0, ns = 1;
  for (int p = 0; p < f.nrad; ++p) {
    const int r = f.radix[p];
    if (r == 4) stockham_pass<4, S>(buf[cur], buf[cur ^ 1], f.tw, f.len, ns);
    else if (r == 2) stockham_pass<2, S>(buf[cur], buf[cur ^ 1], f.tw, f.len, ns);
    else stockham_pass<3, S>(buf[cur], buf[cur ^ 1], f.tw, f.len, ns);
    ns *= r;
    cur ^= 1;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < f.len; i += blockDim.x) base[(long long)i * f.elem_stride] = buf[cur][i];
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

// Add the wave's pupil corrections in slot (= sequence) order and compute
// max |P|^2 over the support.  The support rows are cut into kNormParts
// chunks; chunk c of tile t writes its maximum to pnorm_part[t][c] and readers
// take the max of the kNormParts values, so the result does not depend on
// scheduling.  merge_chunk is one chunk done by one whole CTA.
__device__ __forceinline__ void merge_chunk(float2 *__restrict__ pup, const float2 *__restrict__ dpup,
                                            float *__restrict__ pnorm_part, const int2 *__restrict__ chords, int t,
                                            int ns, int chunk, int y_lo, int rows, int m, int slots) {
  const int rpp = (rows + kNormParts - 1) / kNormParts;
  const int r0 = chunk * rpp, r1 = min(rows, r0 + rpp);
  const size_t mm = (size_t)m * m;
  float2 *p = pup + (size_t)t * mm;
  float mx = 0.f;
  for (int idx = threadIdx.x; idx < (r1 - r0) * m; idx += blockDim.x) {
    const int by = y_lo + r0 + idx / m, bx = idx % m;
    const int2 ch = chords[by];
    if (bx < ch.x || bx > ch.y) continue;
    const size_t off = (size_t)by * m + bx;
    float2 v = p[off];
    if (ns > 0) {
      const float2 *d = dpup + (size_t)t * slots * mm + off;
      int s = 0;
      for (; s + 4 <= ns; s += 4) {
        const float2 a0 = d[(size_t)s * mm], a1 = d[(size_t)(s + 1) * mm];
        const float2 a2 = d[(size_t)(s + 2) * mm], a3 = d[(size_t)(s + 3) * mm];
        v = cadd(cadd(cadd(cadd(v, a0), a1), a2), a3);
      }
      for (; s < ns; ++s) v = cadd(v, d[(size_t)s * mm]);
      p[off] = v;
    }
    mx = fmaxf(mx, cabs2(v));
  }
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __syncthreads();                       // red may still be read by a previous call
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = (threadIdx.x < blockDim.x / 32) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) pnorm_part[(size_t)t * kNormParts + chunk] = v;
  }
}

// Grid: (merge entries (tile, slots), kNormParts chunks).
static __global__ void __launch_bounds__(256) merge_kernel(float2 *__restrict__ pup, const float2 *__restrict__ dpup,
                                                           float *__restrict__ pnorm_part,
                                                           const int2 *__restrict__ merges,
                                                           const int2 *__restrict__ chords, int y_lo, int rows, int m,
                                                           int slots) {
  const int2 mg = merges[blockIdx.x];
  merge_chunk(pup, dpup, pnorm_part, chords, mg.x, mg.y, blockIdx.y, y_lo, rows, m, slots);
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
