// Runtime entry points shared between the host translation units.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "internal.h"
#include "update_args.h"

namespace fpm {
// Twiddle table of the line FFT: exp(sign 2 pi i j / len), j < len.
std::vector<float2> twiddles_line(int len, int sign);
// Line FFTs out of place (src: input at the same offsets, null = in place), with
// an optional finish: output sample e of line l (within its batch) times
// finish * (-1)^(e + l).
int launch_fft_lines_ex(float2 *data, const float2 *src, const float2 *tw, int len, int sign, long long n_lines,
                        int lines_per_batch, long long batch_stride, long long line_stride, long long elem_stride,
                        float finish, cudaStream_t st);
// Row transforms of `tiles` N x N tiles (N = n; tw_pass: the twiddles in pass
// order, FftLines::tw_pass, or null) from src (tiles src_tile_stride
// elements apart) into data (packed, N^2 apart), every row also writing its band
// sums to band[3 l ..]: sum_{x < ov} (-1)^x y_x, sum_{x >= N - ov} (-1)^x y_x and
// its input sample N / 2 (l = tile b's row k at b N + k).
int launch_fft_rows_banded(float2 *data, const float2 *src, const float2 *tw, const float2 *tw_pass, int n, int sign,
                           int tiles, long long src_tile_stride, float2 *band, int ov, cudaStream_t st);
// Column transforms of `tiles` packed N x N tiles (N = n) whose outputs go
// straight into the stitched image: sample (y, x) of packed tile b, which is
// tile t = tile0 + b tile_step of the grid, times finish (-1)^(x+y) and
// weight[t], where the tile keeps row y and column x.
int launch_fft_columns_to_fov(const float2 *data, const float2 *tw, const float2 *tw_pass, int n, int sign, int tiles,
                              float finish, float2 *fov, const float2 *weight, long long fov_w, int ov, int tiles_y,
                              int tiles_x, int tile0, int tile_step, cudaStream_t st);
int launch_fft_lines(float2 *data, const float2 *tw, int len, int sign, long long n_lines, int lines_per_batch,
                     long long batch_stride, long long line_stride, long long elem_stride, cudaStream_t st);
struct QueueJob;
// One persistent launch over several loaded plans (cached per batch).
int run_batch(const std::vector<QueueJob> &jobs, cudaStream_t st, bool graph);
// The same batch run wave by wave, every plan an independent branch (of one cached graph).
int run_batch_waves(const std::vector<QueueJob> &jobs, cudaStream_t st, bool graph);
// Persistent batched execution of `iters` loops of one plan.
int run_persistent(fpm_plan *p, int32_t iters, cudaStream_t st, bool graph, bool stall_test);

// The update-kernel variant for tile side m with `rows` support rows: its
// factorisation m = a * b, cluster size and threads; false if none fits.
bool update_variant(int m, int rows, int *a, int *b, int *cluster, int *threads);
// Twiddle tables of the update kernel's two-pass split m = a * b (m entries each).
void update_twiddles(int m, int a, int b, float2 *inv, float2 *fwd);
// Launch the update kernel over items [item0, item0 + count) (image dtype FPM_U16 or FPM_F32);
// band: the support fits the band, so the variant's band-pruned twin runs where it has one.
int launch_update_items(int m, int rows, int dtype, const UpdateArgs &a, long long item0, long long count,
                        cudaStream_t st, bool band = false);
// The plan's device state (tables, spectra, pupils), created on first use.
int ensure_device_state(fpm_plan *p);
// Free the plan's online-ingestion state, if any (online.cu).
void destroy_online_state(fpm_plan *p);
// Wave steps launched so far by the plan's online ingestion, and in its schedule (0, 0 if none).
void online_progress(const fpm_plan *p, int32_t *launched, int32_t *total);
// The tile-image buffer for images of type dtype, (re)allocated as needed.
int ensure_images(fpm_plan *p, int32_t dtype);
// Gather n_src sensor images (LEDs led0 .. led0 + n_src - 1, planes stride_led
// elements apart) into the tile-image buffer, stream-ordered.
int gather_tile_images(fpm_plan *p, const void *src, int32_t dtype, long long stride_led, long long stride_row,
                       int led0, int n_src, cudaStream_t st);
// Initial guess of every tile from `plane`, the sensor image of the order's first
// LED (rows stride_row elements apart); resets the pupils.  Uses the plan's dtype.
int run_init(fpm_plan *p, const void *plane, long long stride_row, cudaStream_t st);
// Wave steps [s0, s1) captured as one graph of `branches` tile-group branches.
int capture_wave_steps(fpm_plan *p, int32_t iters, int s0, int s1, int branches, cudaGraphExec_t *out);
// Wave steps [s0, s1) of the `iters`-loop schedule, launched as FPM_RUN_WAVES does.
int enqueue_wave_steps(fpm_plan *p, int32_t iters, int s0, int s1, cudaStream_t st);
// Set the plan's image type and intensity scale and clear its error word (before a load).
int begin_load(fpm_plan *p, int32_t dtype, float counts_per_unit, cudaStream_t st);
// Mark the plan loaded (its state is ready for fpm_reconstruct and the getters).
void mark_loaded(fpm_plan *p);
// Validate an image stack description; *bytes (if set) = its extent in bytes.
int validate_stack(fpm_plan *p, const void *stack, int32_t dtype, int64_t stride_led, int64_t stride_row,
                   float counts_per_unit, size_t *bytes);
// fpm_load_tiles without the ownership check (the server loads the plans it owns).
int load_tiles(fpm_plan *p, const void *stack, int32_t dtype, int32_t on_device, int64_t stride_led,
               int64_t stride_row, float counts_per_unit, cudaStream_t st);
// Device bytes of a plan's tile images (the update kernel's column layout) of type dtype.
size_t image_bytes(const fpm_plan *p, int32_t dtype);
// Device bytes a plan takes once loaded with images of type dtype (spectra,
// pupils, corrections and the tile images).
size_t plan_device_bytes(const fpm_plan *p, int32_t dtype);
// Device-side description of a loaded plan for the update kernel (items unset).
UpdateArgs plan_update_args(fpm_plan *p);
// Image element type of a loaded plan (FPM_U16 / FPM_F32); -1 if not loaded.
int plan_image_dtype(const fpm_plan *p);
// The plan's device error word ([0] code, [1] abort flag), or null.
unsigned *plan_error_word(fpm_plan *p);
// The plan's spectra [T][N][N] (centred complex64) once loaded, else null.
const float2 *plan_spectra(const fpm_plan *p);
// Slot of the plan's stitch tables (device memory freed with the plan; null
// until the first stitch builds them), or null without device state.
float2 **plan_stitch_tables(fpm_plan *p);
// Whether the plan's support lies in the band of the band-pruned update kernels.
bool plan_band_fits(const fpm_plan *p);
// The plan's second stream for the stitch and its kStitchEvents events (made on
// first use, destroyed with the plan).
constexpr int kStitchEvents = 5;
int plan_stitch_streams(fpm_plan *p, cudaStream_t *aux, cudaEvent_t **ev);
// A device scratch buffer of at least `bytes`, kept with the plan (grown on
// demand, freed with the plan); its contents do not survive the next call.
int plan_scratch(fpm_plan *p, size_t bytes, void **out);
// Launch the pupil merge over `count` (tile, slots) entries.
int launch_merge(float2 *pup, const float2 *dpup, const int2 *entries, int count, int y_lo, int rows, int m,
                 int slots, int disc, cudaStream_t st);
}  // namespace fpm
