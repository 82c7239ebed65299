// Argument block of the fused per-LED update kernel, shared by the host
// launchers and the kernels.
#pragma once
#include <cuda_runtime.h>

namespace fpm {

// Row chunks of the pupil merge (merge_kernel).
constexpr int kNormParts = 4;

// Image layout read by the update kernel (m = A * B, the kernel's split): for
// tile t and LED l the m x m image is stored column after column, and within
// column x position k1 * B + k2 holds row y = k1 + A * k2, the order in which
// the radix-B pass of the column transform consumes it.  One lane's B pixels
// are then contiguous.
// Half-width bound of the support disc in box row by (support rows y_lo ..
// y_lo + rows - 1, centre column m/2): the support's chord in that row lies in
// [m/2 - hw, m/2 + hw].  With rows = 2 floor(r) + 1 for a disc of radius r,
// r < (rows + 1) / 2, so hw = floor(sqrt(((rows + 1)/2)^2 - dy^2)) + 1 bounds
// the chord; plans verify it against their chords (disc_bound_covers).  Every
// step is exact in float or correctly rounded, so host and device agree.
__host__ __device__ inline int disc_half_width(int by, int y_lo, int rows) {
  const float rr = 0.5f * (float)(rows + 1);
  const float dy = (float)by - ((float)y_lo + 0.5f * (float)(rows - 1));
#ifdef __CUDA_ARCH__
  const float h2 = __fsub_rn(__fmul_rn(rr, rr), __fmul_rn(dy, dy));
#else
  const float h2 = rr * rr - dy * dy;
#endif
  return (int)sqrtf(h2 > 0.f ? h2 : 0.f) + 1;
}

// Band pruning of the update (tile sides whose first pass is radix 16): the
// band is box positions [kBandBlocks B, (A - kBandBlocks) B) in both directions;
// band_fits tells whether a support of rows [y_lo, y_hi] and columns
// [c_lo, c_hi] lies inside it, so that the pruned kernels may run.
constexpr int kBandBlocks = 3;
__host__ __device__ inline bool band_fits(int a, int b, int zb, int y_lo, int y_hi, int c_lo, int c_hi) {
  const int lo = zb * b, hi = (a - zb) * b - 1;
  return y_lo >= lo && y_hi <= hi && c_lo >= lo && c_hi <= hi;
}

// The split of each supported tile side; every kernel for that side uses it.
constexpr int image_split_a(int m) { return m == 64 ? 8 : m == 128 ? 16 : m == 192 ? 12 : m == 256 ? 16 : 0; }
__host__ __device__ inline size_t tile_image_offset(int t, int l, int n_leds, int m) {
  return ((size_t)t * n_leds + l) * (size_t)m * m;
}

struct UpdateArgs {
  float2 *spec;               // [T][N][N] centred spectra
  const float2 *pup;          // [T][m][m] centred pupils (as of the update's wave start)
  float2 *dpup;               // [T][slots][m][m] pupil corrections (EPRY) or null; zero off the support
  const int4 *items;          // (tile, led, slot, sequence index)
  const int2 *shifts;         // [T][L] (sy, sx)
  const int2 *chords;         // [m] (lo, hi) support columns per box row
  const float2 *tw_inv;       // [m] exp(+2 pi i b k1/m) at k1*B + b
  const float2 *tw_fwd;       // [m] exp(-2 pi i b k1/m) at k1*A + b (the B x A split)
  const void *images;         // [T][L][m][m] tile images in the column layout below
  float inv_counts;           // intensity = element * inv_counts
  float scale;                // (N/m)^2
  int n;                      // N
  int n_leds;
  int y_lo;                   // first support row (box coordinates)
  int rows;                   // R
  int slots;                  // correction slots per tile
  int disc;                   // 1: disc_half_width bounds every support chord
  unsigned *err;
};

}  // namespace fpm
