// Argument block of the fused per-LED update kernel, shared by the host
// launchers and the kernels.
#pragma once
#include <cuda_runtime.h>

namespace fpm {

// Row chunks of the pupil merge (merge_kernel).
constexpr int kNormParts = 8;

struct UpdateArgs {
  float2 *spec;               // [T][N][N] centred spectra
  const float2 *pup;          // [T][m][m] centred pupils (as of the update's wave start)
  float2 *dpup;               // [T][slots][m][m] pupil corrections (EPRY) or null; zero off the support
  const int4 *items;          // (tile, led, slot, sequence index)
  const int2 *shifts;         // [T][L] (sy, sx)
  const int2 *origins;        // [T] (y0, x0) on the sensor
  const int2 *chords;         // [m] (lo, hi) support columns per box row
  const float2 *tw_inv;       // [m] exp(+2 pi i b k1/m) at k1*B + b
  const float2 *tw_fwd;       // [m] exp(-2 pi i b k1/m) at k1*A + b (the B x A split)
  const void *stack;          // images, element (l, y, x) at l*stride_led + y*stride_row + x
  long long stride_led, stride_row;
  float inv_counts;           // intensity = element * inv_counts
  float scale;                // (N/m)^2
  int n;                      // N
  int n_leds;
  int y_lo;                   // first support row (box coordinates)
  int rows;                   // R
  int slots;                  // correction slots per tile
  unsigned *err;
};

}  // namespace fpm
