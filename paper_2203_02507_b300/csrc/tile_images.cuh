// Gather of the image stack into the update kernel's tile-major column layout.
#pragma once
#include <cuda_runtime.h>

#include "update_args.h"

namespace fpm {

// Tile images in the update kernel's column layout (tile_image_offset):
// out[t][led0 + l][x][k1 * b + k2] = stack[l][y0_t + k1 + a k2][x0_t + x] for
// the n_src images l of `stack` (LEDs led0 .. led0 + n_src - 1 of n_leds).  One
// block per (tile, image, 32 columns): the block reads the 32 columns row by
// row into shared memory (pitch 33 words) and writes them out column by column.
// Shared memory: m * 33 * 4 bytes.
template <typename Img>
__global__ void tile_images_kernel(Img *out, const Img *stack, long long stride_led, long long stride_row,
                                   const int2 *origins, int m, int a, int b, int n_leds, int led0, int n_src,
                                   long long n_blocks) {
  extern __shared__ unsigned col_buf[];
  const int chunks = m / 32;
  for (long long blk = blockIdx.x; blk < n_blocks; blk += gridDim.x) {
    const int chunk = (int)(blk % chunks);
    const int l = (int)((blk / chunks) % n_src);
    const int t = (int)(blk / ((long long)chunks * n_src));
    const int x0 = chunk * 32;
    const int2 o = origins[t];
    const Img *src = stack + (long long)l * stride_led + (long long)o.x * stride_row + o.y + x0;
    __syncthreads();   // the previous block's reads of col_buf are done
    // kLoads independent loads per thread in flight before their shared-memory stores
    constexpr int kLoads = 16;
    for (int i0 = threadIdx.x; i0 < m * 32; i0 += blockDim.x * kLoads) {
      Img v[kLoads];
#pragma unroll
      for (int u = 0; u < kLoads; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i < m * 32) v[u] = src[(long long)(i >> 5) * stride_row + (i & 31)];
      }
#pragma unroll
      for (int u = 0; u < kLoads; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i < m * 32) {
          if constexpr (sizeof(Img) == 2) col_buf[(i >> 5) * 33 + (i & 31)] = (unsigned)v[u];
          else col_buf[(i >> 5) * 33 + (i & 31)] = __float_as_uint(v[u]);
        }
      }
    }
    __syncthreads();
    Img *dst = out + tile_image_offset(t, led0 + l, n_leds, m) + (size_t)x0 * m;
    for (int i = threadIdx.x; i < m * 32; i += blockDim.x) {
      const int x = i / m, j = i - x * m;
      const int y = j / b + a * (j % b);
      const unsigned v = col_buf[y * 33 + x];
      if constexpr (sizeof(Img) == 2) dst[(size_t)x * m + j] = (Img)v;
      else dst[(size_t)x * m + j] = __uint_as_float(v);
    }
  }
}

}  // namespace fpm
