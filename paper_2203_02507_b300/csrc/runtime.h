// Runtime entry points shared between the host translation units.
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace fpm {
int launch_fft_lines(float2 *data, const float2 *tw, int len, int sign, long long n_lines, int lines_per_batch,
                     long long batch_stride, long long line_stride, long long elem_stride, cudaStream_t st);
// Persistent batched execution of `iters` loops of one plan (persistent.cu).
int run_persistent(fpm_plan *p, int32_t iters, cudaStream_t st, bool graph);
}  // namespace fpm
