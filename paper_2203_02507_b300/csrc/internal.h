// Internal declarations shared by the host-side translation units of libfpm.
#pragma once

#include <cstdint>
#include <deque>
#include <string>
#include <vector>

#include "../../include/fpm.h"

namespace fpm {

// Set the calling thread's error text and return `code`.
int fail(int code, const char *fmt, ...);
void clear_error();

struct DeviceState;   // device-side buffers of a plan (runtime.cu)
struct OnlineState;   // image-by-image ingestion of a plan (online.cu)

// Wave-step work lists of a plan's schedule, flattened for launches.  Step s
// holds wave s of every tile that has one.
struct StepLists {
  // item = (tile, led, slot, sequence index); items of step s are
  // items[step_off[s] .. step_off[s+1]), sorted by tile
  std::vector<int32_t> items;       // 4 ints per item
  std::vector<int64_t> step_off;    // [n_steps + 1]
  // merges of step s: (tile, n_slots) in merges[merge_off[s] .. merge_off[s+1])
  std::vector<int32_t> merges;      // 2 ints per entry
  std::vector<int64_t> merge_off;   // [n_steps + 1]
  int32_t n_steps = 0;
  int32_t iters = 0;                // prefix of the sequence these lists cover
};

}  // namespace fpm

struct fpm_plan {
  // problem statement (copied)
  int32_t sensor_h = 0, sensor_w = 0, m = 0, overlap = 0, tiles_y = 0, tiles_x = 0;
  int32_t upsample = 0, n = 0, n_tiles = 0, n_leds = 0, iters = 0, order_kind = 0;
  double wavelength_um = 0, na = 0, pixel_um = 0, led_height_um = 0, df = 0;
  bool epry = false;
  bool sequential = false;          // FPM_SEQUENTIAL: one update per wave
  bool unmasked = false;            // FPM_EPRY_UNMASKED: updates over the whole m x m box
  std::vector<double> led_xy, defocus;
  // tile subset (Sec. 5, sub-regions sent to different GPUs): this plan holds
  // tiles [tile_first, tile_first + n_tiles) of the tiles_y x tiles_x grid
  // (row-major); subset = false when it holds the whole grid
  int32_t tile_first = 0;
  bool subset = false;

  // data-independent quantities (host, FP64 -> int / complex64)
  std::vector<int32_t> origins;     // [T][2] (y0, x0)
  std::vector<int32_t> shifts;      // [T][L][2] (sy, sx)
  std::vector<int32_t> order;       // [L]
  std::vector<int32_t> waves;       // [T][iters * L]
  std::vector<int32_t> n_waves;     // [T]
  std::vector<uint8_t> support;     // [m][m] where updates act (the circular pupil support,
                                    // or the whole box with FPM_EPRY_UNMASKED)
  std::vector<uint8_t> circ;        // [m][m] the circular pupil support (initial pupils)
  std::vector<int32_t> chord_lo, chord_hi;   // [m], per box row; lo > hi when empty
  int32_t y_lo = 0, y_hi = -1;      // support rows (box coordinates)
  bool disc_ok = false;             // disc_half_width bounds every chord
  bool band_ok = false;             // the support lies in the band-pruned update's band
  int32_t support_px = 0;
  int32_t max_waves = 0, max_width = 0;
  int64_t total_waves = 0;
  std::vector<float> pupil0;        // [T][m][m][2]

  // launch configuration of the update kernel (chosen at plan time)
  int32_t cluster = 1, threads = 256;

  fpm::DeviceState *dev = nullptr;
  fpm::OnlineState *online = nullptr;
  int32_t busy = 0;                 // > 0 while a server job owns the plan

  // cached step lists keyed by iteration count
  std::deque<fpm::StepLists> step_cache;   // deque: references stay valid as it grows
};

namespace fpm {
// Circular pupil support |f| <= NA / wavelength on the m x m centred grid,
// f = (b - m/2) * df: per box row the inclusive column range [lo, hi] (lo > hi
// when empty) and the first/last support rows.  Returns the pixel count, or -1
// when a row is not one contiguous chord or the rows are not contiguous.
// lo/hi (and mask, if not null) must hold m (m * m) entries.
int support_chords(int m, double df, double na, double wavelength_um, uint8_t *mask, int32_t *lo, int32_t *hi,
                   int32_t *y_lo, int32_t *y_hi);
// True if disc_half_width (the kernels' table-free chord bound) covers every
// support chord [lo[by], hi[by]], by in [y_lo, y_hi].
bool disc_bound_covers(int m, int32_t y_lo, int32_t y_hi, const int32_t *lo, const int32_t *hi);
// Build (or fetch from the cache) the wave-step lists for the first `iters` loops.
const StepLists &step_lists(fpm_plan *p, int32_t iters);
// Free device state (runtime.cu).
void destroy_device_state(fpm_plan *p);
// Choose cluster size and threads for (m, support rows); returns false if nothing fits.
bool choose_launch(int32_t m, int32_t rows, int32_t *cluster, int32_t *threads);
}  // namespace fpm
