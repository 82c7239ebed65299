// Stitching of the reconstructed tiles into one high-resolution field of view
// (Eq. 1, Sec. 3.1), and the per-tile object behind it.
//
// Object of a tile: o = IDFT_N(ifftshift O) with the 1/N^2 factor.  With O in
// centred storage (frequency k - N/2 at index k) this is (-1)^(x+y) / N^2 times
// the unnormalised inverse transform of O taken in natural order, so the
// spectra are transformed along rows (out of place) and columns by the line FFT,
// the column pass applying the sign and scale as it stores.
//
// Stitching follows Eq. 1 pairwise: each column of tiles top to bottom (part 1),
// then the columns left to right (part 2).  Output line i < r - ov/2 of a pair
// is the first image's, later lines are the second image's times mu1 / mu2, the
// complex means of the two images over the ov lines they share (ov = LR overlap
// times the upsampling).  Because every output pixel comes from exactly one
// tile, the whole sequence reduces to one complex weight per tile:
//   part 1, column j:  c(0,j) = 1,  c(i,j) = c(i-1,j) B(i-1,j) / T(i,j)
//   part 2:            d(0) = 1,   d(j) = d(j-1) SR(j-1) / SL(j)
// with T/B the sums of a tile over its first/last ov rows, and SL/SR the sums of
// a column image over its first/last ov columns, SL(j) = sum_i c(i,j) L(i,j),
// L(i,j) the sum of tile (i,j) over its first ov columns and the rows it keeps
// in its column image (likewise R over the last ov columns).  The band sums are
// reduced on the device in a fixed order (FP64 across threads), the weights
// chained on the host in FP64, and one pass writes every output pixel as
// weight x object.  A zero denominator (or ov = 0: no shared band) gives
// weight 1, as in Eq. 1's reading for a dark band.
#include <cuda_runtime.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "internal.h"
#include "runtime.h"

namespace fpm {

#define FPM_CK(call)                                                                         \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(FPM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Row range [r0, r1) that tile row i keeps in its column image of K tiles.
__host__ __device__ inline void kept_rows(int i, int k_tiles, int n, int ov, int *r0, int *r1) {
  *r0 = i > 0 ? ov - ov / 2 : 0;
  *r1 = i < k_tiles - 1 ? n - ov / 2 : n;
}

// Band sums of every tile in a fixed order: grid (tiles, 4, kBandChunks),
// band 0 = first ov rows, 1 = last ov rows, 2 = first ov columns over the kept
// rows, 3 = last ov columns over the kept rows; chunk z sums the z-th of
// kBandChunks consecutive parts of the band.
// out[(t * 4 + band) * kBandChunks + z] = (re, im); the host adds the chunks in order.
constexpr int kBandThreads = 256, kBandChunks = 16;
static __global__ void __launch_bounds__(kBandThreads) band_sums_kernel(const float2 *obj, int n, int ov,
                                                                        int tiles_y, int tiles_x, double2 *out) {
  __shared__ double sre[kBandThreads], sim[kBandThreads];
  const int t = blockIdx.x, band = blockIdx.y, z = blockIdx.z;
  const int i = t / tiles_x;
  int y0 = 0, y1 = n, x0 = 0, x1 = n;
  if (band == 0) y1 = ov;
  if (band == 1) y0 = n - ov;
  if (band >= 2) {
    kept_rows(i, tiles_y, n, ov, &y0, &y1);
    if (band == 2) x1 = ov;
    else x0 = n - ov;
  }
  // chunk z: rows [y0 + z rows / kBandChunks, ...) of the band, columns [x0, x1)
  const int rows = y1 - y0;
  const int ya = y0 + rows * z / kBandChunks, yb = y0 + rows * (z + 1) / kBandChunks;
  const float2 *o = obj + (size_t)t * n * n;
  // a thread's few dozen samples in FP32 (FP64 arithmetic is slow on this part),
  // the block's partials combined in FP64; the threads stride over the chunk's
  // samples row after row, so narrow column bands keep every thread busy
  float re = 0.f, im = 0.f;
  const int width = x1 - x0, count = (yb - ya) * width;
#pragma unroll 4
  for (int i = (int)threadIdx.x; i < count; i += kBandThreads) {
    const int y = ya + i / width, x = x0 + i % width;
    const float2 v = o[(size_t)y * n + x];
    re += v.x;
    im += v.y;
  }
  sre[threadIdx.x] = (double)re;
  sim[threadIdx.x] = (double)im;
  __syncthreads();
  for (int s = kBandThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sre[threadIdx.x] += sre[threadIdx.x + s];
      sim[threadIdx.x] += sim[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[((size_t)t * 4 + band) * kBandChunks + z] = make_double2(sre[0], sim[0]);
}

// Tile (row or column) index of field-of-view line X: tile 0 up to
// n - ov/2, then one tile per stride n - ov.
__device__ __forceinline__ int tile_of_line(int x, int n, int ov, int k_tiles) {
  if (x < n - ov / 2) return 0;
  return min(k_tiles - 1, 1 + (x - (n - ov / 2)) / (n - ov));
}

// out[X][Y] = weight(i, j) * object(i, j)[X - i (n - ov)][Y - j (n - ov)]; rows X
// strided over the grid, columns over the threads of a block.
static __global__ void assemble_kernel(float2 *out, const float2 *obj, const float2 *weight, int n, int ov,
                                       int tiles_y, int tiles_x, int fov_h, int fov_w) {
  const int stride = n - ov;
  for (int x = blockIdx.x; x < fov_h; x += gridDim.x) {
    const int i = tile_of_line(x, n, ov, tiles_y);
    const float2 *orow = obj + (size_t)i * tiles_x * n * n + (size_t)(x - i * stride) * n;
    float2 *dst = out + (size_t)x * fov_w;
    for (int y = threadIdx.x; y < fov_w; y += blockDim.x) {
      const int j = tile_of_line(y, n, ov, tiles_x);
      const float2 v = orow[(size_t)j * n * n + (y - j * stride)];
      const float2 wt = weight[i * tiles_x + j];
      dst[y] = make_float2(__fmaf_rn(wt.x, v.x, -__fmul_rn(wt.y, v.y)), __fmaf_rn(wt.x, v.y, __fmul_rn(wt.y, v.x)));
    }
  }
}

}  // namespace fpm

namespace fpm {

struct StitchGeom {
  int n = 0, ov = 0, ty = 0, tx = 0, fov_h = 0, fov_w = 0;
};

static StitchGeom stitch_geom(const fpm_plan *p) {
  StitchGeom g;
  g.n = p->n;
  g.ov = p->overlap * p->upsample;
  g.ty = p->tiles_y;
  g.tx = p->tiles_x;
  g.fov_h = g.n + (g.ty - 1) * (g.n - g.ov);
  g.fov_w = g.n + (g.tx - 1) * (g.n - g.ov);
  return g;
}

static unsigned grid_of(long long work, int threads) {
  return (unsigned)std::max<long long>(1, std::min<long long>((work + threads - 1) / threads, 148LL * 32));
}

// Objects of tiles [t0, t0 + count) into buf (count x N x N), stream-ordered: the
// row transforms read the spectra and write buf, the column transforms run in
// place and apply (-1)^(x+y) / N^2 as they store.
static int tile_objects(const fpm_plan *p, int t0, int count, float2 *buf, const float2 *tw_inv_n, cudaStream_t st) {
  const int n = p->n;
  const size_t nn = (size_t)n * n;
  int rc;
  if ((rc = launch_fft_lines_ex(buf, plan_spectra(p) + (size_t)t0 * nn, tw_inv_n, n, +1, (long long)count * n, n,
                                (long long)nn, n, 1, 0.f, st)))
    return rc;
  return launch_fft_lines_ex(buf, nullptr, tw_inv_n, n, +1, (long long)count * n, n, (long long)nn, 1, n,
                             (float)(1.0 / ((double)n * n)), st);
}

static int check_loaded(const fpm_plan *p) {
  if (!plan_spectra(p)) return fail(FPM_ESTATE, "no spectra before fpm_load_tiles");
  if (p->busy) return fail(FPM_EBUSY, "plan is owned by a server job");
  return FPM_OK;
}

// A run whose bounded device wait gave up leaves no valid state to read.
static int check_device_error(fpm_plan *p, cudaStream_t st) {
  unsigned *err = plan_error_word(p);
  unsigned e = 0;
  FPM_CK(cudaStreamSynchronize(st));
  if (err) FPM_CK(cudaMemcpy(&e, err, sizeof(e), cudaMemcpyDeviceToHost));
  if (e) return fail(FPM_ETIMEOUT, "a bounded device wait of the last persistent run gave up");
  return FPM_OK;
}

// Per-tile weights of the stitched image from the band sums (see the top of the file).
static std::vector<float2> stitch_weights(const StitchGeom &g, const std::vector<double2> &sums) {
  using cd = std::complex<double>;
  const int T = g.ty * g.tx;
  std::vector<cd> c(T, cd(1.0, 0.0)), d(g.tx, cd(1.0, 0.0));
  auto sum = [&](int t, int band) {
    cd v(0.0, 0.0);
    for (int z = 0; z < kBandChunks; ++z) {
      const double2 c = sums[((size_t)t * 4 + band) * kBandChunks + z];
      v += cd(c.x, c.y);
    }
    return v;
  };
  if (g.ov > 0) {
    for (int j = 0; j < g.tx; ++j)
      for (int i = 1; i < g.ty; ++i) {
        const int t = i * g.tx + j, up = (i - 1) * g.tx + j;
        const cd top = sum(t, 0);
        c[t] = top != cd(0.0, 0.0) ? c[up] * sum(up, 1) / top : cd(1.0, 0.0);
      }
    for (int j = 1; j < g.tx; ++j) {
      cd sl(0.0, 0.0), sr(0.0, 0.0);
      for (int i = 0; i < g.ty; ++i) {
        sl += c[i * g.tx + j] * sum(i * g.tx + j, 2);
        sr += c[i * g.tx + j - 1] * sum(i * g.tx + j - 1, 3);
      }
      d[j] = sl != cd(0.0, 0.0) ? d[j - 1] * sr / sl : cd(1.0, 0.0);
    }
  }
  std::vector<float2> w(T);
  for (int t = 0; t < T; ++t) {
    const cd v = c[t] * d[t % g.tx];
    w[t] = make_float2((float)v.real(), (float)v.imag());
  }
  return w;
}

}  // namespace fpm

using fpm::fail;

namespace {
// Consecutive 256-byte aligned pieces of one scratch buffer.
struct Carve {
  size_t off = 0;
  template <class T>
  size_t take(size_t count) {
    const size_t at = off;
    off = (off + count * sizeof(T) + 255) & ~size_t(255);
    return at;
  }
};
}  // namespace

extern "C" {

int fpm_get_object(fpm_plan *p, int32_t tile, void *dst, int32_t on_device, void *stream) {
  fpm::clear_error();
  if (!p || !dst) return fail(FPM_EINVAL, "fpm_get_object: null argument");
  if (tile < 0 || tile >= p->n_tiles) return fail(FPM_EINVAL, "tile %d out of range", tile);
  int rc = fpm::check_loaded(p);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nn = (size_t)p->n * p->n;
  Carve cv;
  const size_t o_buf = cv.take<float2>(nn), o_tw = cv.take<float2>(p->n);
  void *base = nullptr;
  if ((rc = fpm::plan_scratch(p, cv.off, &base))) return rc;
  float2 *buf = reinterpret_cast<float2 *>(static_cast<char *>(base) + o_buf);
  float2 *tw = reinterpret_cast<float2 *>(static_cast<char *>(base) + o_tw);
  const std::vector<float2> twh = fpm::twiddles_line(p->n, +1);
  if (cudaMemcpyAsync(tw, twh.data(), twh.size() * sizeof(float2), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return fail(FPM_ECUDA, "fpm_get_object: table upload failed");
  if ((rc = fpm::tile_objects(p, tile, 1, buf, tw, st))) return rc;
  if (cudaMemcpyAsync(dst, buf, nn * sizeof(float2), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                      st) != cudaSuccess)
    return fail(FPM_ECUDA, "fpm_get_object: copy out failed");
  return on_device ? FPM_OK : fpm::check_device_error(p, st);
}

int fpm_stitch(fpm_plan *p, void *dst, int32_t on_device, void *stream) {
  fpm::clear_error();
  if (!p || !dst) return fail(FPM_EINVAL, "fpm_stitch: null argument");
  if (p->subset) return fail(FPM_EINVAL, "fpm_stitch needs a plan of the whole tile grid (this one holds a subset)");
  int rc = fpm::check_loaded(p);
  if (rc) return rc;
  const fpm::StitchGeom g = fpm::stitch_geom(p);
  if (g.ov < 0 || 2 * g.ov > g.n)
    return fail(FPM_EINVAL, "HR overlap %d: stitching needs 0 <= overlap <= N/2 = %d", g.ov, g.n / 2);
  cudaStream_t st = (cudaStream_t)stream;
  const int T = p->n_tiles;
  const size_t nn = (size_t)g.n * g.n, fov = (size_t)g.fov_h * g.fov_w;
  Carve cv;
  const size_t o_obj = cv.take<float2>((size_t)T * nn), o_tw = cv.take<float2>(g.n);
  const size_t o_sums = cv.take<double2>((size_t)T * 4 * fpm::kBandChunks), o_w = cv.take<float2>(T);
  const size_t o_out = on_device ? 0 : cv.take<float2>(fov);
  void *base = nullptr;
  if ((rc = fpm::plan_scratch(p, cv.off, &base))) return rc;
  char *b = static_cast<char *>(base);
  float2 *obj = reinterpret_cast<float2 *>(b + o_obj), *tw = reinterpret_cast<float2 *>(b + o_tw);
  double2 *sums = reinterpret_cast<double2 *>(b + o_sums);
  float2 *wdev = reinterpret_cast<float2 *>(b + o_w);
  float2 *out = on_device ? static_cast<float2 *>(dst) : reinterpret_cast<float2 *>(b + o_out);
  const std::vector<float2> twh = fpm::twiddles_line(g.n, +1);
  if (cudaMemcpyAsync(tw, twh.data(), twh.size() * sizeof(float2), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return fail(FPM_ECUDA, "fpm_stitch: table upload failed");
  if ((rc = fpm::tile_objects(p, 0, T, obj, tw, st))) return rc;
  std::vector<double2> sh((size_t)T * 4 * fpm::kBandChunks, make_double2(0.0, 0.0));
  if (g.ov > 0) {
    fpm::band_sums_kernel<<<dim3((unsigned)T, 4, fpm::kBandChunks), fpm::kBandThreads, 0, st>>>(obj, g.n, g.ov, g.ty,
                                                                                                 g.tx, sums);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(sh.data(), sums, sh.size() * sizeof(double2), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(FPM_ECUDA, "fpm_stitch: band sums failed");
  }
  const std::vector<float2> w = fpm::stitch_weights(g, sh);
  if (cudaMemcpyAsync(wdev, w.data(), w.size() * sizeof(float2), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return fail(FPM_ECUDA, "fpm_stitch: weight upload failed");
  fpm::assemble_kernel<<<(unsigned)std::min(g.fov_h, 148 * 32), 256, 0, st>>>(out, obj, wdev, g.n, g.ov, g.ty, g.tx,
                                                                             g.fov_h, g.fov_w);
  if (cudaGetLastError() != cudaSuccess) return fail(FPM_ECUDA, "fpm_stitch: assembly launch failed");
  if (!on_device && cudaMemcpyAsync(dst, out, fov * sizeof(float2), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail(FPM_ECUDA, "fpm_stitch: copy out failed");
  return on_device ? FPM_OK : fpm::check_device_error(p, st);
}

}  // extern "C"
