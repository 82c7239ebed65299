// Host-side planning: validation, FP64 geometry, LED order, pupils and the
// dependency-levelled wave schedule.  No CUDA call is made in this file.
//
// Geometry follows Sec. 2.2 (an LED is a point source; every sub-region sees
// it at its own angle) and Sec. 3.1 (overlapping square sub-regions).  The
// wave schedule is the spectrum-domain parallelism of Sec. 3.2: updates whose
// sub-aperture discs share no spectrum pixel may run together, across
// iteration loops.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>

#include "internal.h"
#include "update_args.h"

namespace fpm {

static thread_local std::string g_error;

int fail(int code, const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_error = buf;
  return code;
}

void clear_error() { g_error.clear(); }

// C lround semantics (halfway cases away from zero), on a finite double.
static inline int64_t round_half_away(double v) { return (int64_t)std::lround(v); }

// Run f(i) for i in [0, n) on up to hardware_concurrency threads.
template <class F>
static void parallel_for(int64_t n, F f) {
  unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  int64_t nt = std::min<int64_t>(n, (int64_t)std::min(hw, 32u));
  if (nt <= 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  for (int64_t k = 0; k < nt; ++k)
    th.emplace_back([=, &f]() {
      for (int64_t i = k; i < n; i += nt) f(i);
    });
  for (auto &t : th) t.join();
}

bool disc_bound_covers(int m, int32_t y_lo, int32_t y_hi, const int32_t *lo, const int32_t *hi) {
  const int rows = y_hi - y_lo + 1;
  for (int by = y_lo; by <= y_hi; ++by) {
    const int hw = disc_half_width(by, y_lo, rows);
    if (lo[by] > hi[by]) continue;
    if (lo[by] < std::max(0, m / 2 - hw) || hi[by] > std::min(m - 1, m / 2 + hw)) return false;
  }
  return true;
}

int support_chords(int m, double df, double na, double wavelength_um, uint8_t *mask, int32_t *lo_v, int32_t *hi_v,
                   int32_t *y_lo, int32_t *y_hi) {
  for (int i = 0; i < m; ++i) {
    lo_v[i] = 1;
    hi_v[i] = 0;
  }
  const double cutoff = na / wavelength_um;
  int count = 0;
  *y_lo = m;
  *y_hi = -1;
  for (int by = 0; by < m; ++by) {
    const double fy = (double)(by - m / 2) * df;
    int lo = m, hi = -1, in_row = 0;
    for (int bx = 0; bx < m; ++bx) {
      const double fx = (double)(bx - m / 2) * df;
      const bool in = std::sqrt(fx * fx + fy * fy) <= cutoff;
      if (mask) mask[(size_t)by * m + bx] = in;
      if (in) {
        lo = std::min(lo, bx);
        hi = std::max(hi, bx);
        ++count;
        ++in_row;
      }
    }
    if (hi >= lo) {
      if (in_row != hi - lo + 1) return -1;                 // rows must be chords
      lo_v[by] = lo;
      hi_v[by] = hi;
      *y_lo = std::min(*y_lo, by);
      *y_hi = std::max(*y_hi, by);
    }
  }
  for (int by = *y_lo; by <= *y_hi; ++by)
    if (hi_v[by] < lo_v[by]) return -1;                      // rows must be contiguous
  return count;
}

static bool build_support(fpm_plan *p) {
  p->support.assign((size_t)p->m * p->m, 0);
  p->chord_lo.assign(p->m, 1);
  p->chord_hi.assign(p->m, 0);
  const int c = support_chords(p->m, p->df, p->na, p->wavelength_um, p->support.data(), p->chord_lo.data(),
                               p->chord_hi.data(), &p->y_lo, &p->y_hi);
  p->disc_ok = c > 0 && disc_bound_covers(p->m, p->y_lo, p->y_hi, p->chord_lo.data(), p->chord_hi.data());
  p->support_px = c > 0 ? c : 0;
  p->circ = p->support;
  if (c > 0 && p->unmasked) {
    // unmasked EPRY: spectrum and pupil corrections, normalisers and footprints
    // over the whole box; the initial pupil keeps the circular support
    std::fill(p->support.begin(), p->support.end(), (uint8_t)1);
    for (int by = 0; by < p->m; ++by) {
      p->chord_lo[by] = 0;
      p->chord_hi[by] = p->m - 1;
    }
    p->y_lo = 0;
    p->y_hi = p->m - 1;
    p->disc_ok = false;
    p->support_px = p->m * p->m;
  }
  // band pruning: rows and every chord inside the band of the first radix-16 pass
  const int a = image_split_a(p->m);
  p->band_ok = false;
  if (c > 0 && a == 16) {
    int c_lo = p->m, c_hi = -1;
    for (int by = p->y_lo; by <= p->y_hi; ++by) {
      c_lo = std::min(c_lo, p->chord_lo[by]);
      c_hi = std::max(c_hi, p->chord_hi[by]);
    }
    p->band_ok = band_fits(a, p->m / a, kBandBlocks, p->y_lo, p->y_hi, c_lo, c_hi);
  }
  return c > 0;
}

static void build_pupils(fpm_plan *p) {
  const int m = p->m;
  p->pupil0.assign((size_t)p->n_tiles * m * m * 2, 0.f);
  const double inv_l = 1.0 / p->wavelength_um;
  for (int t = 0; t < p->n_tiles; ++t) {
    const double z = p->defocus.empty() ? 0.0 : p->defocus[t];
    float *dst = p->pupil0.data() + (size_t)t * m * m * 2;
    for (int by = 0; by < m; ++by) {
      const double fy = (double)(by - m / 2) * p->df;
      for (int bx = 0; bx < m; ++bx) {
        if (!p->circ[(size_t)by * m + bx]) continue;
        const double fx = (double)(bx - m / 2) * p->df;
        const double f2 = fx * fx + fy * fy;
        const double kz = std::sqrt(std::max(inv_l * inv_l - f2, 0.0)) - inv_l;
        const double ph = 2.0 * M_PI * z * kz;
        dst[((size_t)by * m + bx) * 2 + 0] = (float)std::cos(ph);
        dst[((size_t)by * m + bx) * 2 + 1] = (float)std::sin(ph);
      }
    }
  }
}

static void build_geometry(fpm_plan *p) {
  const int m = p->m, T = p->n_tiles, L = p->n_leds;
  const int stride = m - p->overlap;
  const int span_y = (p->tiles_y - 1) * stride + m;
  const int span_x = (p->tiles_x - 1) * stride + m;
  const int my = (p->sensor_h - span_y) / 2, mx = (p->sensor_w - span_x) / 2;
  p->origins.resize((size_t)T * 2);
  for (int i = 0; i < p->tiles_y; ++i)
    for (int j = 0; j < p->tiles_x; ++j) {
      p->origins[(size_t)(i * p->tiles_x + j) * 2 + 0] = my + i * stride;
      p->origins[(size_t)(i * p->tiles_x + j) * 2 + 1] = mx + j * stride;
    }
  p->shifts.resize((size_t)T * L * 2);
  const double h = p->led_height_um;
  for (int t = 0; t < T; ++t) {
    const double yc = ((double)p->origins[t * 2 + 0] + m / 2.0 - p->sensor_h / 2.0) * p->pixel_um;
    const double xc = ((double)p->origins[t * 2 + 1] + m / 2.0 - p->sensor_w / 2.0) * p->pixel_um;
    for (int l = 0; l < L; ++l) {
      const double dx = p->led_xy[(size_t)l * 2 + 0] - xc;
      const double dy = p->led_xy[(size_t)l * 2 + 1] - yc;
      const double r = std::sqrt(dx * dx + dy * dy + h * h);
      const double u = dx / r, v = dy / r;
      p->shifts[((size_t)t * L + l) * 2 + 0] = (int32_t)round_half_away(v / (p->wavelength_um * p->df));
      p->shifts[((size_t)t * L + l) * 2 + 1] = (int32_t)round_half_away(u / (p->wavelength_um * p->df));
    }
  }
  // LED order (Sec. 3.2): centre-out = by squared distance from the axis, ties by index.
  p->order.resize(L);
  for (int l = 0; l < L; ++l) p->order[l] = l;
  if (p->order_kind == FPM_ORDER_CENTER_OUT) {
    std::vector<double> d2(L);
    for (int l = 0; l < L; ++l) {
      const double x = p->led_xy[(size_t)l * 2], y = p->led_xy[(size_t)l * 2 + 1];
      d2[l] = x * x + y * y;
    }
    std::stable_sort(p->order.begin(), p->order.end(),
                     [&](int a, int b) { return d2[a] < d2[b]; });
  }
}

// Waves.  Two updates conflict when their support discs, centred at c + s_a and
// c + s_b, share an HR pixel, i.e. when d = s_b - s_a is in the difference set
// {k - k' : k, k' in support}.  Because every update conflicts with the
// previous update of the same LED, the largest wave among the earlier updates
// of LED b is the wave of its latest update; so
//   wave(j) = 1 + max over LEDs b conflicting with LED(j) of last_wave[b]
// (0 when there is none), which is the definition over all earlier updates.
static void build_waves(fpm_plan *p) {
  const int m = p->m, T = p->n_tiles, L = p->n_leds, S = p->iters * L;
  const int R = p->y_hi - p->y_lo + 1;
  int wmax = 0;
  for (int by = p->y_lo; by <= p->y_hi; ++by) wmax = std::max(wmax, p->chord_hi[by] - p->chord_lo[by] + 1);
  // conflict table over d in [-(R-1), R-1] x [-(wmax-1), wmax-1]
  const int DY = R - 1, DX = wmax - 1;
  const int dw = 2 * DX + 1;
  std::vector<uint8_t> conflict((size_t)(2 * DY + 1) * dw, 0);
  for (int dy = -DY; dy <= DY; ++dy)
    for (int dx = -DX; dx <= DX; ++dx) {
      bool hit = false;
      // exists row y with y and y - dy both support rows, chords overlapping after +dx
      for (int y = p->y_lo; y <= p->y_hi && !hit; ++y) {
        const int y2 = y - dy;
        if (y2 < p->y_lo || y2 > p->y_hi) continue;
        const int lo = std::max(p->chord_lo[y], p->chord_lo[y2] + dx);
        const int hi = std::min(p->chord_hi[y], p->chord_hi[y2] + dx);
        hit = lo <= hi;
      }
      conflict[(size_t)(dy + DY) * dw + (dx + DX)] = hit;
    }
  (void)m;
  p->waves.assign((size_t)T * S, 0);
  p->n_waves.assign(T, 0);
  std::vector<int32_t> widths_max(T, 0);
  parallel_for(T, [&](int64_t t) {
    const int32_t *sh = p->shifts.data() + (size_t)t * L * 2;
    std::vector<std::vector<int32_t>> nbr(L);
    for (int a = 0; a < L; ++a)
      for (int b = 0; b < L; ++b) {
        const int dy = sh[b * 2] - sh[a * 2], dx = sh[b * 2 + 1] - sh[a * 2 + 1];
        if (dy < -DY || dy > DY || dx < -DX || dx > DX) continue;
        if (conflict[(size_t)(dy + DY) * dw + (dx + DX)]) nbr[a].push_back(b);
      }
    std::vector<int32_t> last(L, -1);
    int32_t *w = p->waves.data() + (size_t)t * S;
    int32_t top = -1;
    for (int j = 0; j < S; ++j) {
      const int l = p->order[j % L];
      int32_t mx = -1;
      if (p->sequential) {
        mx = j - 1;                      // strict sequence: one update per wave
      } else {
        for (int b : nbr[l]) mx = std::max(mx, last[b]);
      }
      w[j] = mx + 1;
      last[l] = mx + 1;
      top = std::max(top, mx + 1);
    }
    p->n_waves[t] = top + 1;
    std::vector<int32_t> cnt(top + 1, 0);
    for (int j = 0; j < S; ++j) ++cnt[w[j]];
    widths_max[t] = *std::max_element(cnt.begin(), cnt.end());
  });
  p->max_waves = 0;
  p->max_width = 0;
  p->total_waves = 0;
  for (int t = 0; t < T; ++t) {
    p->max_waves = std::max(p->max_waves, p->n_waves[t]);
    p->max_width = std::max(p->max_width, widths_max[t]);
    p->total_waves += p->n_waves[t];
  }
}

const StepLists &step_lists(fpm_plan *p, int32_t iters) {
  for (auto &s : p->step_cache)
    if (s.iters == iters) return s;
  const int T = p->n_tiles, L = p->n_leds, S = p->iters * L, Sp = iters * L;
  StepLists sl;
  sl.iters = iters;
  int32_t steps = 0;
  for (int t = 0; t < T; ++t) {
    const int32_t *w = p->waves.data() + (size_t)t * S;
    for (int j = 0; j < Sp; ++j) steps = std::max(steps, w[j] + 1);
  }
  sl.n_steps = steps;
  // counting sort of (step, tile, j)
  std::vector<int64_t> per_step(steps + 1, 0);
  for (int t = 0; t < T; ++t) {
    const int32_t *w = p->waves.data() + (size_t)t * S;
    for (int j = 0; j < Sp; ++j) ++per_step[w[j] + 1];
  }
  for (int s = 0; s < steps; ++s) per_step[s + 1] += per_step[s];
  sl.step_off = per_step;
  sl.items.assign((size_t)per_step[steps] * 4, 0);
  std::vector<int64_t> fill(per_step.begin(), per_step.end() - 1);
  std::vector<std::vector<int32_t>> merge_step(steps);
  std::vector<int32_t> slot(steps, 0);
  for (int t = 0; t < T; ++t) {
    const int32_t *w = p->waves.data() + (size_t)t * S;
    std::fill(slot.begin(), slot.end(), 0);
    for (int j = 0; j < Sp; ++j) {
      const int s = w[j];
      int32_t *it = sl.items.data() + (size_t)fill[s]++ * 4;
      it[0] = t;
      it[1] = p->order[j % L];
      it[2] = slot[s]++;
      it[3] = j;
    }
    for (int s = 0; s < steps; ++s)
      if (slot[s] > 0) {
        merge_step[s].push_back(t);
        merge_step[s].push_back(slot[s]);
      }
  }
  sl.merge_off.assign(steps + 1, 0);
  for (int s = 0; s < steps; ++s) {
    sl.merge_off[s + 1] = sl.merge_off[s] + (int64_t)merge_step[s].size() / 2;
    sl.merges.insert(sl.merges.end(), merge_step[s].begin(), merge_step[s].end());
  }
  p->step_cache.push_back(std::move(sl));
  return p->step_cache.back();
}

}  // namespace fpm

using fpm::fail;

extern "C" {

const char *fpm_last_error(void) { return fpm::g_error.c_str(); }

int fpm_plan_create(const fpm_plan_desc *d, fpm_plan **out) {
  fpm::clear_error();
  if (!d || !out) return fail(FPM_EINVAL, "fpm_plan_create: null argument");
  *out = nullptr;
  const int m = d->tile;
  if (m != 64 && m != 128 && m != 192 && m != 256)
    return fail(FPM_EINVAL, "tile side %d not supported (64, 128, 192 or 256)", m);
  if (d->upsample < 2 || d->upsample > 8)
    return fail(FPM_EINVAL, "upsample %d out of range [2, 8]", d->upsample);
  if (d->tiles_y < 1 || d->tiles_x < 1 || d->tiles_y > 4096 || d->tiles_x > 4096)
    return fail(FPM_EINVAL, "tile grid %d x %d out of range", d->tiles_y, d->tiles_x);
  if (d->overlap < 0 || d->overlap >= m)
    return fail(FPM_EINVAL, "overlap %d must be in [0, tile)", d->overlap);
  if (d->sensor_h < m || d->sensor_w < m)
    return fail(FPM_EINVAL, "sensor %d x %d smaller than a tile", d->sensor_h, d->sensor_w);
  const int stride = m - d->overlap;
  if ((int64_t)(d->tiles_y - 1) * stride + m > d->sensor_h ||
      (int64_t)(d->tiles_x - 1) * stride + m > d->sensor_w)
    return fail(FPM_EINVAL, "tile grid does not fit the sensor");
  if (!(d->wavelength_um > 0) || !(d->na > 0) || !(d->na < 1) || !(d->pixel_um > 0) ||
      !(d->led_height_um > 0) || !std::isfinite(d->wavelength_um) || !std::isfinite(d->pixel_um) ||
      !std::isfinite(d->led_height_um))
    return fail(FPM_EINVAL, "optics must be positive and finite (0 < NA < 1)");
  if (d->n_leds < 1 || d->n_leds > 65536 || !d->led_xy_um)
    return fail(FPM_EINVAL, "need 1..65536 LEDs with positions");
  if (d->iters < 1 || d->iters > 10000) return fail(FPM_EINVAL, "iters %d out of range", d->iters);
  if (d->order != FPM_ORDER_CENTER_OUT && d->order != FPM_ORDER_RASTER)
    return fail(FPM_EINVAL, "unknown order %d", d->order);
  if (d->flags & ~(FPM_EPRY | FPM_SEQUENTIAL | FPM_EPRY_UNMASKED)) return fail(FPM_EINVAL, "unknown flags 0x%x", d->flags);
  const int64_t grid_tiles = (int64_t)d->tiles_y * d->tiles_x;
  if (d->tile_first < 0 || d->tile_count < 0 || (int64_t)d->tile_first + d->tile_count > grid_tiles ||
      (d->tile_count == 0 && d->tile_first != 0))
    return fail(FPM_EINVAL, "tile subset [%d, %d + %d) outside the %lld tiles of the grid", d->tile_first,
                d->tile_first, d->tile_count, (long long)grid_tiles);
  if ((d->flags & FPM_EPRY_UNMASKED) && !(d->flags & FPM_EPRY))
    return fail(FPM_EINVAL, "FPM_EPRY_UNMASKED needs FPM_EPRY");

  fpm_plan *p = new (std::nothrow) fpm_plan();
  if (!p) return fail(FPM_ENOMEM, "out of host memory");
  p->sensor_h = d->sensor_h;
  p->sensor_w = d->sensor_w;
  p->m = m;
  p->overlap = d->overlap;
  p->tiles_y = d->tiles_y;
  p->tiles_x = d->tiles_x;
  p->upsample = d->upsample;
  p->n = d->upsample * m;
  p->n_tiles = d->tiles_y * d->tiles_x;
  p->n_leds = d->n_leds;
  p->iters = d->iters;
  p->order_kind = d->order;
  p->wavelength_um = d->wavelength_um;
  p->na = d->na;
  p->pixel_um = d->pixel_um;
  p->led_height_um = d->led_height_um;
  p->epry = (d->flags & FPM_EPRY) != 0;
  p->sequential = (d->flags & FPM_SEQUENTIAL) != 0;
  p->unmasked = (d->flags & FPM_EPRY_UNMASKED) != 0;
  p->df = 1.0 / (m * d->pixel_um);
  p->led_xy.assign(d->led_xy_um, d->led_xy_um + (size_t)d->n_leds * 2);
  for (double v : p->led_xy)
    if (!std::isfinite(v)) {
      delete p;
      return fail(FPM_EINVAL, "LED positions must be finite");
    }
  if (d->defocus_um) {
    p->defocus.assign(d->defocus_um, d->defocus_um + p->n_tiles);
    for (double v : p->defocus)
      if (!std::isfinite(v)) {
        delete p;
        return fail(FPM_EINVAL, "defocus must be finite");
      }
  }
  if (!fpm::build_support(p)) {
    delete p;
    return fail(FPM_EINVAL, "pupil support is empty or not a disc on the %d x %d grid", m, m);
  }
  const int rows = p->y_hi - p->y_lo + 1;
  if (!fpm::choose_launch(m, rows, &p->cluster, &p->threads)) {
    delete p;
    return fail(FPM_EINVAL, "pupil support (%d rows) too large for tile %d: NA*m*pixel/wavelength too big", rows, m);
  }
  fpm::build_geometry(p);
  if (d->tile_count > 0 && d->tile_count < grid_tiles) {   // keep the subset's tiles only
    const int f = d->tile_first, c = d->tile_count, L = p->n_leds;
    p->origins.erase(p->origins.begin(), p->origins.begin() + (size_t)f * 2);
    p->origins.resize((size_t)c * 2);
    p->shifts.erase(p->shifts.begin(), p->shifts.begin() + (size_t)f * L * 2);
    p->shifts.resize((size_t)c * L * 2);
    if (!p->defocus.empty()) {
      p->defocus.erase(p->defocus.begin(), p->defocus.begin() + f);
      p->defocus.resize(c);
    }
    p->n_tiles = c;
    p->tile_first = f;
    p->subset = true;
  }
  // every sub-aperture box must stay inside the N x N spectrum
  for (int t = 0; t < p->n_tiles; ++t)
    for (int l = 0; l < p->n_leds; ++l) {
      const int64_t y0 = p->n / 2 + (int64_t)p->shifts[((size_t)t * p->n_leds + l) * 2] - m / 2;
      const int64_t x0 = p->n / 2 + (int64_t)p->shifts[((size_t)t * p->n_leds + l) * 2 + 1] - m / 2;
      if (y0 < 0 || x0 < 0 || y0 + m > p->n || x0 + m > p->n) {
        const int sy = p->shifts[((size_t)t * p->n_leds + l) * 2], sx = p->shifts[((size_t)t * p->n_leds + l) * 2 + 1];
        delete p;
        return fail(FPM_EINVAL, "tile %d LED %d: sub-aperture shift (%d, %d) leaves the %d x %d spectrum", t, l, sy, sx,
                    m * d->upsample, m * d->upsample);
      }
    }
  fpm::build_pupils(p);
  fpm::build_waves(p);
  *out = p;
  return FPM_OK;
}

int fpm_plan_destroy(fpm_plan *p) {
  if (!p) return FPM_OK;
  if (p->busy) return fail(FPM_EBUSY, "plan is owned by a server job");
  fpm::destroy_device_state(p);
  delete p;
  return FPM_OK;
}

int fpm_plan_get_info(const fpm_plan *p, fpm_plan_info *info) {
  if (!p || !info) return fail(FPM_EINVAL, "fpm_plan_get_info: null argument");
  std::memset(info, 0, sizeof(*info));
  info->m = p->m;
  info->n = p->n;
  info->n_tiles = p->n_tiles;
  info->n_leds = p->n_leds;
  info->iters = p->iters;
  info->support_px = p->support_px;
  info->support_rows = p->y_hi - p->y_lo + 1;
  info->max_waves = p->max_waves;
  info->max_wave_width = p->max_width;
  info->total_waves = p->total_waves;
  const int64_t T = p->n_tiles, n = p->n, m = p->m;
  info->device_bytes = T * n * n * 8 + T * m * m * 8 * (p->epry ? 2 + p->max_width : 2);
  info->cluster = p->cluster;
  info->threads = p->threads;
  info->image_elems = T * p->n_leds * m * m;
  info->hr_overlap = p->overlap * p->upsample;
  info->fov_h = (int32_t)(n + (p->tiles_y - 1) * (n - info->hr_overlap));
  info->fov_w = (int32_t)(n + (p->tiles_x - 1) * (n - info->hr_overlap));
  info->tile_first = p->tile_first;
  info->band = p->band_ok ? 1 : 0;
  return FPM_OK;
}

int fpm_get_schedule(const fpm_plan *p, int32_t *order, int32_t *shifts, int32_t *waves, int32_t *origins) {
  if (!p) return fail(FPM_EINVAL, "fpm_get_schedule: null plan");
  if (order) std::memcpy(order, p->order.data(), p->order.size() * 4);
  if (shifts) std::memcpy(shifts, p->shifts.data(), p->shifts.size() * 4);
  if (waves) std::memcpy(waves, p->waves.data(), p->waves.size() * 4);
  if (origins) std::memcpy(origins, p->origins.data(), p->origins.size() * 4);
  return FPM_OK;
}

int fpm_initial_pupil(const fpm_plan *p, int32_t tile, void *dst) {
  if (!p || !dst) return fail(FPM_EINVAL, "fpm_initial_pupil: null argument");
  if (tile < 0 || tile >= p->n_tiles) return fail(FPM_EINVAL, "tile %d out of range", tile);
  const size_t mm = (size_t)p->m * p->m;
  std::memcpy(dst, p->pupil0.data() + (size_t)tile * mm * 2, mm * 8);
  return FPM_OK;
}

}  // extern "C"
