// Runtime entry points shared between the host translation units.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "internal.h"
#include "update_args.h"

namespace fpm {
int launch_fft_lines(float2 *data, const float2 *tw, int len, int sign, long long n_lines, int lines_per_batch,
                     long long batch_stride, long long line_stride, long long elem_stride, cudaStream_t st);
// Persistent batched execution of `iters` loops of one plan (persistent.cu).
int run_persistent(fpm_plan *p, int32_t iters, cudaStream_t st, bool graph);

// The update-kernel variant for tile side m with `rows` support rows: its
// factorisation m = a * b, cluster size and threads; false if none fits.
bool update_variant(int m, int rows, int *a, int *b, int *cluster, int *threads);
// Twiddle tables of the update kernel's two-pass split m = a * b (m entries each).
void update_twiddles(int m, int a, int b, float2 *inv, float2 *fwd);
// Launch the update kernel over items [item0, item0 + count) (image dtype FPM_U16 or FPM_F32).
int launch_update_items(int m, int rows, int dtype, const UpdateArgs &a, long long item0, long long count,
                        cudaStream_t st);
// Launch the pupil merge / normaliser over `count` (tile, slots) entries.
int launch_merge(float2 *pup, const float2 *dpup, float *pnorm_part, const int2 *merges, int count,
                 const int2 *chords, int y_lo, int rows, int m, int slots, cudaStream_t st);
}  // namespace fpm
