// Gather of the image stack into the update kernel's tile-major column layout.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "update_args.h"

namespace fpm {

// Tile images in the update kernel's column layout (tile_image_offset):
// out[t][led0 + l][x][k1 * B + k2] = stack[l][y0_t + k1 + A k2][x0_t + x] for
// the n_src images l of `stack` (LEDs led0 .. led0 + n_src - 1 of n_leds), with
// A = image_split_a(M), B = M / A.  One block per (tile, image, 32 columns):
// the block reads the 32 columns row by row into shared memory (pitch 33
// words, conflict-free both ways) and writes them out column by column.
//
// Both sides move 16-byte words: a row segment of 32 pixels is 4 (16-bit) or 8
// (32-bit) words, and since B is a multiple of the pixels per word, a word of
// the output holds pixels of one k1 and consecutive k2.  `vec` says that the
// stack's base and strides are 16-byte aligned; a tile whose column origin is
// not on a 16-byte boundary reads its rows pixel by pixel instead.  The output
// is always aligned (tile images are whole multiples of 16 bytes).
// Shared memory: M * 33 * 4 bytes.
template <typename Img, int M>
__global__ void __launch_bounds__(256) tile_images_kernel(Img *out, const Img *stack, long long stride_led,
                                                          long long stride_row, const int2 *origins, int n_leds,
                                                          int led0, int n_src, long long n_blocks, int vec) {
  constexpr int A = image_split_a(M), B = M / A;
  constexpr int V = 16 / (int)sizeof(Img);           // pixels per 16-byte word
  constexpr int RW = 32 / V;                          // words per 32-pixel row segment
  constexpr int LOADS = M * RW / 256;                 // words per thread, load side
  constexpr int STORES = 32 * (M / V) / 256;          // words per thread, store side
  static_assert(A > 0 && B % V == 0, "a 16-byte output word holds one k1 and consecutive k2");
  static_assert(M * RW % 256 == 0 && 32 * (M / V) % 256 == 0, "whole words per thread");
  extern __shared__ unsigned col_buf[];
  constexpr int chunks = M / 32;
  for (long long blk = blockIdx.x; blk < n_blocks; blk += gridDim.x) {
    const int chunk = (int)(blk % chunks);
    const int l = (int)((blk / chunks) % n_src);
    const int t = (int)(blk / ((long long)chunks * n_src));
    const int x0 = chunk * 32;
    const int2 o = origins[t];
    const Img *src = stack + (long long)l * stride_led + (long long)o.x * stride_row + o.y + x0;
    __syncthreads();   // the previous block's reads of col_buf are done
    if (vec && (o.y % V) == 0) {
      uint4 w[LOADS];
#pragma unroll
      for (int u = 0; u < LOADS; ++u) {               // all loads in flight first
        const int k = threadIdx.x + u * 256;
        const int y = k / RW, c = k % RW;
        w[u] = __ldg(reinterpret_cast<const uint4 *>(src + (long long)y * stride_row) + c);
      }
#pragma unroll
      for (int u = 0; u < LOADS; ++u) {
        const int k = threadIdx.x + u * 256;
        const int y = k / RW, c = k % RW;
        unsigned *row = col_buf + y * 33 + c * V;
        const unsigned q[4] = {w[u].x, w[u].y, w[u].z, w[u].w};
#pragma unroll
        for (int e = 0; e < V; ++e) {
          if constexpr (sizeof(Img) == 2) row[e] = (q[e >> 1] >> (16 * (e & 1))) & 0xffffu;
          else row[e] = q[e];
        }
      }
    } else {
      constexpr int kLoads = 16;
      for (int i0 = threadIdx.x; i0 < M * 32; i0 += 256 * kLoads) {
        Img v[kLoads];
#pragma unroll
        for (int u = 0; u < kLoads; ++u) {
          const int i = i0 + u * 256;
          if (i < M * 32) v[u] = src[(long long)(i >> 5) * stride_row + (i & 31)];
        }
#pragma unroll
        for (int u = 0; u < kLoads; ++u) {
          const int i = i0 + u * 256;
          if (i < M * 32) {
            if constexpr (sizeof(Img) == 2) col_buf[(i >> 5) * 33 + (i & 31)] = (unsigned)v[u];
            else col_buf[(i >> 5) * 33 + (i & 31)] = __float_as_uint(v[u]);
          }
        }
      }
    }
    __syncthreads();
    uint4 *dst = reinterpret_cast<uint4 *>(out + tile_image_offset(t, led0 + l, n_leds, M) + (size_t)x0 * M);
#pragma unroll
    for (int u = 0; u < STORES; ++u) {
      // consecutive threads write consecutive words of one output column
      const int k = threadIdx.x + u * 256;
      const int x = k / (M / V), jw = k % (M / V);
      const int j0 = jw * V, k1 = j0 / B, k20 = j0 % B;
      unsigned q[4];
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const unsigned v = col_buf[(k1 + A * (k20 + e)) * 33 + x];
        if constexpr (sizeof(Img) == 2) {
          if (e & 1) q[e >> 1] |= v << 16;
          else q[e >> 1] = v;
        } else {
          q[e] = v;
        }
      }
      dst[(size_t)x * (M / V) + jw] = make_uint4(q[0], q[1], q[2], q[3]);
    }
  }
}

// Launch of tile_images_kernel for tile side m (64, 128, 192 or 256) over
// n_tiles tiles and n_src images; returns the launch status.
template <typename Img>
inline cudaError_t launch_tile_images(Img *out, const Img *stack, long long stride_led, long long stride_row,
                                      const int2 *origins, int m, int n_tiles, int n_leds, int led0, int n_src,
                                      cudaStream_t st) {
  const long long n_blocks = (long long)n_tiles * n_src * (m / 32);
  if (n_blocks <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)(n_blocks < 148LL * 6 * 4 ? n_blocks : 148LL * 6 * 4);
  const size_t smem = (size_t)m * 33 * sizeof(unsigned);
  const int es = (int)sizeof(Img);
  const int vec = ((uintptr_t)stack % 16 == 0) && (stride_row * es) % 16 == 0 && (stride_led * es) % 16 == 0;
  switch (m) {
    case 64:
      tile_images_kernel<Img, 64><<<grid, 256, smem, st>>>(out, stack, stride_led, stride_row, origins, n_leds, led0,
                                                           n_src, n_blocks, vec);
      break;
    case 128:
      tile_images_kernel<Img, 128><<<grid, 256, smem, st>>>(out, stack, stride_led, stride_row, origins, n_leds, led0,
                                                            n_src, n_blocks, vec);
      break;
    case 192:
      tile_images_kernel<Img, 192><<<grid, 256, smem, st>>>(out, stack, stride_led, stride_row, origins, n_leds, led0,
                                                            n_src, n_blocks, vec);
      break;
    case 256:
      tile_images_kernel<Img, 256><<<grid, 256, smem, st>>>(out, stack, stride_led, stride_row, origins, n_leds, led0,
                                                            n_src, n_blocks, vec);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fpm
