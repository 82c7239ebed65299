// One LED update of one tile that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a host whose device memory is entirely
// reserved by its own pool allocator, a plug-in that may not allocate after
// start-up, or a real-time acquisition loop in which an allocation (and the
// device synchronisation that cudaMalloc/cudaFree can imply) would stall the
// camera.  fpm_update_tile_static serves them: the caller passes the spectrum,
// the pupil and the measured image, and every temporary the update needs (the
// pupil correction, the support chords, the twiddle tables, the one-item work
// list, the merge entry and the image rearranged into the update kernel's
// column layout) lives in the file-scope array below.
//
// The array is a fixed 1 MiB per device that loads this library, held until
// the process exits.  All calls on a device share it and it keeps the last
// call's contents; every byte a call reads is first written by that same call
// (nothing has to start at zero), and calls that overlap on the GPU (different
// streams, or different host threads without ordering) race on it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "runtime.h"
#include "tile_images.cuh"

namespace fpm {

constexpr size_t kStaticScratchBytes = size_t(1) << 20;

static __device__ __align__(256) unsigned char g_fpm_static_scratch[kStaticScratchBytes];

// Host side: the array's device address.  It is looked up (cudaGetSymbolAddress,
// with the device current) on the first call made on a device, and again
// whenever that device's current context is not the one the address was taken
// in (after cudaDeviceReset a new primary context loads the module afresh, so
// an address cached from the old context would dangle).  The context is named
// by its process-unique id, read through the driver entry points the runtime
// hands out, so the library links no driver library of its own.
constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static void *g_scratch_addr[kMaxDevices] = {};
static unsigned long long g_scratch_ctx[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Process-unique id of the calling thread's current context; 0 if it cannot be read.
static unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    cudaGetLastError();
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

static int scratch_address(int dev, void **out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(FPM_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  // cudaFree(0) makes the device's primary context current, so the id read next
  // is the context the address below belongs to
  cudaError_t e = cudaFree(nullptr);
  if (e != cudaSuccess) return fail(FPM_ECUDA, "initialising device %d: %s", dev, cudaGetErrorString(e));
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fpm_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(FPM_ECUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_addr[dev];
  return FPM_OK;
}

// True when p is device (or managed) memory of device `dev`, the device the
// kernels of this call run on.  Memory of another GPU is refused: without peer
// access the kernels could not reach it.
static bool is_device_pointer(const void *p, int dev) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace fpm

using fpm::fail;

extern "C" int fpm_update_tile_static(void *spectrum, int32_t n, void *pupil, int32_t m, const float *image,
                                      int32_t shift_y, int32_t shift_x, double wavelength_um, double na,
                                      double pixel_um, int32_t epry, void *stream) {
  fpm::clear_error();
  if (!spectrum || !pupil || !image) return fail(FPM_EINVAL, "fpm_update_tile_static: null argument");
  if (m < 16 || m > 4096 || m % 16) return fail(FPM_EINVAL, "tile side %d out of range", m);
  if (n < 2 * m || n > 8 * m || n % m)
    return fail(FPM_EINVAL, "HR side %d must be 2..8 times the tile side %d", n, m);
  // layout of the static array: [pupil correction m*m][tables][image in the kernel's column layout]
  const size_t dp_bytes = (size_t)m * m * sizeof(float2);
  const size_t blob_off = fpm::align256(dp_bytes);
  const size_t chords_b = (size_t)m * sizeof(int2), tw_b = (size_t)m * sizeof(float2);
  const size_t blob_bytes = chords_b + 2 * tw_b + sizeof(int4) + 2 * sizeof(int2) + sizeof(int2);
  const size_t img_off = fpm::align256(blob_off + blob_bytes);
  const size_t need = img_off + (size_t)m * m * sizeof(float);
  if (need > fpm::kStaticScratchBytes)
    return fail(FPM_EINVAL, "tile side %d needs %zu bytes of static scratch; the limit is %zu", m, need,
                fpm::kStaticScratchBytes);
  if (m != 64 && m != 128 && m != 192 && m != 256)
    return fail(FPM_EINVAL, "tile side %d not supported (64, 128, 192 or 256)", m);
  if (!(wavelength_um > 0) || !(na > 0) || !(na < 1) || !(pixel_um > 0))
    return fail(FPM_EINVAL, "optics must be positive (0 < NA < 1)");
  const int64_t oy = n / 2 + (int64_t)shift_y - m / 2, ox = n / 2 + (int64_t)shift_x - m / 2;
  if (oy < 0 || ox < 0 || oy + m > n || ox + m > n)
    return fail(FPM_EINVAL, "shift (%d, %d) moves the %d x %d box out of the %d x %d spectrum", shift_y, shift_x, m,
                m, n, n);
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return fail(FPM_EINVAL, "spectrum, pupil and image must be device memory (no CUDA device)");
  }
  if (!fpm::is_device_pointer(spectrum, cur) || !fpm::is_device_pointer(pupil, cur) ||
      !fpm::is_device_pointer(image, cur))
    return fail(FPM_EINVAL, "spectrum, pupil and image must be device memory of the current device %d", cur);

  // support chords, FP64, exactly as the plan computes them
  int32_t lo[256], hi[256], y_lo = 0, y_hi = -1;
  const double df = 1.0 / (m * pixel_um);
  if (fpm::support_chords(m, df, na, wavelength_um, nullptr, lo, hi, &y_lo, &y_hi) <= 0)
    return fail(FPM_EINVAL, "pupil support is empty or not a disc");
  const int rows = y_hi - y_lo + 1;
  int fa = 0, fb = 0, fc = 0, ft = 0;
  if (!fpm::update_variant(m, rows, &fa, &fb, &fc, &ft))
    return fail(FPM_EINVAL, "pupil support (%d rows) too large for tile %d", rows, m);

  void *base = nullptr;
  int rc = fpm::scratch_address(cur, &base);
  if (rc) return rc;
  unsigned char *dev = static_cast<unsigned char *>(base);

  // tables, built on the stack and copied with one stream-ordered copy
  alignas(16) unsigned char blob[256 * 8 + 2 * 256 * 8 + 64];
  unsigned char *w = blob;
  int2 *ch = reinterpret_cast<int2 *>(w);
  for (int i = 0; i < m; ++i) ch[i] = make_int2(lo[i], hi[i]);
  w += chords_b;
  float2 *twi = reinterpret_cast<float2 *>(w);
  float2 *twf = twi + m;
  fpm::update_twiddles(m, fa, fb, twi, twf);
  w += 2 * tw_b;
  int4 *item = reinterpret_cast<int4 *>(w);
  *item = make_int4(0, 0, 0, 0);         // tile 0, LED 0, slot 0
  int2 *sh = reinterpret_cast<int2 *>(item + 1);
  sh[0] = make_int2(shift_y, shift_x);   // shift of LED 0
  sh[1] = make_int2(0, 0);               // origin of tile 0 in the image
  sh[2] = make_int2(0, 1);               // merge entry: tile 0, one correction
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(dev + blob_off, blob, blob_bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(FPM_ECUDA, "copy of the update tables: %s", cudaGetErrorString(e));

  const int2 *d_chords = reinterpret_cast<const int2 *>(dev + blob_off);
  const float2 *d_twi = reinterpret_cast<const float2 *>(dev + blob_off + chords_b);
  const float2 *d_twf = d_twi + m;
  const int4 *d_item = reinterpret_cast<const int4 *>(dev + blob_off + chords_b + 2 * tw_b);
  const int2 *d_sh = reinterpret_cast<const int2 *>(d_item + 1);
  const int2 *d_mg = d_sh + 2;
  float2 *d_dp = reinterpret_cast<float2 *>(dev);
  float *d_img = reinterpret_cast<float *>(dev + img_off);
  float2 *pup = static_cast<float2 *>(pupil);

  // 0. the image in the update kernel's column layout
  e = fpm::launch_tile_images(d_img, image, (long long)m * m, m, d_sh + 1, m, 1, 1, 0, 1, st);
  if (e != cudaSuccess) return fail(FPM_ECUDA, "image layout: %s", cudaGetErrorString(e));

  // 1. zero the correction (the merge sums whole pixel pairs, so entries off this
  //    call's support must be zero)  2. the update  3. (EPRY) add the correction
  if (epry) {
    e = cudaMemsetAsync(d_dp, 0, dp_bytes, st);
    if (e != cudaSuccess) return fail(FPM_ECUDA, "clearing the static correction: %s", cudaGetErrorString(e));
  }
  fpm::UpdateArgs a{};
  a.spec = static_cast<float2 *>(spectrum);
  a.pup = pup;
  a.dpup = epry ? d_dp : nullptr;
  a.items = d_item;
  a.shifts = d_sh;
  a.chords = d_chords;
  a.tw_inv = d_twi;
  a.tw_fwd = d_twf;
  a.images = d_img;
  a.inv_counts = 1.f;
  a.scale = (float)((double)n / m * (double)n / m);
  a.n = n;
  a.n_leds = 1;
  a.y_lo = y_lo;
  a.rows = rows;
  a.slots = 1;
  a.disc = fpm::disc_bound_covers(m, y_lo, y_hi, lo, hi) ? 1 : 0;
  a.err = nullptr;
  // the band-pruned update where the support fits its band, as a plan would run it
  int c_lo = m, c_hi = -1;
  for (int by = y_lo; by <= y_hi; ++by) {
    c_lo = std::min(c_lo, lo[by]);
    c_hi = std::max(c_hi, hi[by]);
  }
  const bool band = fa == 16 && fpm::band_fits(fa, fb, fpm::kBandBlocks, y_lo, y_hi, c_lo, c_hi);
  if ((rc = fpm::launch_update_items(m, rows, FPM_F32, a, 0, 1, st, band))) return rc;
  const int disc = a.disc;
  if (epry && (rc = fpm::launch_merge(pup, d_dp, d_mg, 1, y_lo, rows, m, 1, disc, st))) return rc;
  return FPM_OK;
}
