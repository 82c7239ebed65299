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
// in its column image (likewise R over the last ov columns).  A zero
// denominator (or ov = 0: no shared band) gives weight 1, as in Eq. 1's reading
// for a dark band.
//
// The band sums need no object: the sum of o over rows Y and columns X is
//   (1/N^2) sum_ky g_Y(ky) sum_kx O[ky][kx] h_X(kx),  g_Y(k) = sum_{y in Y} e^{2 pi i (k - N/2) y / N}
// (likewise h_X), where the inner sum is sum_{x in X} (-1)^x R[ky][x], R the
// natural-order inverse row transform of O, and for X = all columns it is
// N O[ky][N/2].  So the row transforms of a tile give its band values per row
// as they store, and the sums over ky with the closed-form g take a few
// thousand terms per tile.  Weight c(i,j) needs only tiles above (i,j) and d(j)
// only columns up to j, so the tiles go one tile column at a time: row
// transforms into a buffer the size of one tile column (the spectra are read and
// the image written with evict-first hints, so the buffer's lines stay in L2),
// the column's weights on the device, then the column transforms write weight x
// object straight into the stitched image, only where the tile keeps the pixel.
// Two such buffers let the row transforms of column j + 1 run on the caller's
// stream while the weights and column transforms of column j run on a second
// one.  Every spectrum is read once and every image pixel written once; no host
// round trip.
#include <cuda_runtime.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "aux_kernels.cuh"
#include "internal.h"
#include "runtime.h"

namespace fpm {

#define FPM_CK(call)                                                                         \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(FPM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Complex FP32 division by the textbook formula (|b|^2 > 0 checked by the caller).
__device__ __forceinline__ float2 cdiv(float2 a, float2 b) {
  const float r = __frcp_rn(__fadd_rn(__fmul_rn(b.x, b.x), __fmul_rn(b.y, b.y)));
  return make_float2(__fmul_rn(__fadd_rn(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)), r),
                     __fmul_rn(__fsub_rn(__fmul_rn(a.y, b.x), __fmul_rn(a.x, b.y)), r));
}
__device__ __forceinline__ bool cnonzero(float2 a) { return a.x != 0.f || a.y != 0.f; }

// Host tables of a stitch (built once per plan, FP64 rounded to FP32), laid out
//   [0, n)                 tw[j] = e^{+2 pi i j / n}, the inverse line FFT's twiddles
//   [n, n + 1008)          the same twiddles in pass order (FftLines::tw_pass; n = 256, 1024)
//   [n + 1008, 7 n + 1008) g[6][n]: g over the first ov rows, the last ov rows and
//                          the rows kept by the four kept-row classes (class bit 0:
//                          not the first tile row, bit 1: not the last)
constexpr int kPassTab = 240 + 3 * 256;
static std::vector<float2> stitch_tables(int n, int ov) {
  using cd = std::complex<double>;
  std::vector<float2> tab((size_t)7 * n + kPassTab, make_float2(0.f, 0.f));
  const std::vector<float2> tw = twiddles_line(n, +1);
  std::copy(tw.begin(), tw.end(), tab.begin());
  if (n == 256 || n == 1024) {
    float2 *pt = tab.data() + n;
    for (int r = 1; r < 16; ++r)
      for (int k = 0; k < 16; ++k) pt[(r - 1) * 16 + k] = tw[(size_t)k * r * (n / 256)];
    if (n == 1024)
      for (int r = 1; r < 4; ++r)
        for (int j = 0; j < 256; ++j) pt[240 + (r - 1) * 256 + j] = tw[(size_t)j * r];
  }
  // e^{2 pi i j / n} and 1 - e^{2 pi i j / n} (= 2 sin^2(th/2) - i sin th), j reduced exactly
  auto unit = [&](long long j) {
    const long long r = ((j % n) + n) % n;
    const double th = 2.0 * M_PI * (double)r / n;
    return cd(std::cos(th), std::sin(th));
  };
  auto one_minus = [&](long long j) {
    const long long r = ((j % n) + n) % n;
    const double th = 2.0 * M_PI * (double)r / n, sh = std::sin(0.5 * th);
    return cd(2.0 * sh * sh, -std::sin(th));
  };
  // sum_{y0 <= y < y1} e^{2 pi i f y / n}, f = k - n/2: a geometric series
  auto series = [&](int k, int y0, int y1) {
    const long long f = k - n / 2, len = y1 - y0;
    cd v(0.0, 0.0);
    if (len > 0) v = (f % n == 0) ? cd((double)len, 0.0) : unit(f * y0) * one_minus(f * len) / one_minus(f);
    return make_float2((float)v.real(), (float)v.imag());
  };
  float2 *g = tab.data() + n + kPassTab;
  for (int k = 0; k < n; ++k) {
    g[k] = series(k, 0, ov);
    g[(size_t)n + k] = series(k, n - ov, n);
    for (int cls = 0; cls < 4; ++cls) {
      const int y0 = (cls & 1) ? ov - ov / 2 : 0, y1 = (cls & 2) ? n - ov / 2 : n;
      g[(size_t)(2 + cls) * n + k] = series(k, y0, y1);
    }
  }
  return tab;
}

// Band sums and weights of tile column j (grid ty CTAs, kWeightThreads each;
// dynamic shared memory 5 ty float2 for the chain).  CTA i forms the four band
// sums of tile t = i tx + j from its rows' band values (band[3 (i N + ky) ..] =
// r_L(ky), r_R(ky), O[ky][N/2], written by the row transforms):
//   sums[4t + 0] = (1/N)   sum_ky O[ky][N/2] g_top(ky)     (first ov rows)
//   sums[4t + 1] = (1/N)   sum_ky O[ky][N/2] g_bot(ky)     (last ov rows)
//   sums[4t + 2] = (1/N^2) sum_ky r_L(ky) g_kept(ky)       (first ov columns, kept rows)
//   sums[4t + 3] = (1/N^2) sum_ky r_R(ky) g_kept(ky)       (last ov columns, kept rows)
// each thread's terms in order, then a fixed shuffle tree.  The last CTA to
// finish chains the weights on its first warp: the ratios B(r-1) / T(r) in
// parallel, the running product c in row order, the products c L and c R in
// parallel summed by a fixed tree, and d(j) from d(j-1) and SR(j-1) kept in
// colst from the previous column.  All in FP32: the sums carry FP32 rounding
// (about 1e-6 relative) already, and the few chained products and quotients
// add well below that.
constexpr int kWeightThreads = 512;
static __global__ void __launch_bounds__(kWeightThreads)
    stitch_weights_kernel(const float2 *band, const float2 *g, int n, int ty, int tx, int j, float2 *sums,
                          float2 *colst, unsigned *counter, float2 *w) {
  extern __shared__ float2 chain_sm[];              // the column's sums, then its c values
  __shared__ float2 part[kWeightThreads / 32][4];
  __shared__ bool last;
  const int i = blockIdx.x, t = i * tx + j;
  const int cls = (i > 0 ? 1 : 0) | (i < ty - 1 ? 2 : 0);
  const float2 *g_top = g, *g_bot = g + n, *g_kept = g + (size_t)(2 + cls) * n;
  float2 acc[4];
  for (int b = 0; b < 4; ++b) acc[b] = make_float2(0.f, 0.f);
  for (int ky = threadIdx.x; ky < n; ky += kWeightThreads) {
    const float2 *bv = band + 3 * ((size_t)i * n + ky);
    const float2 rl = bv[0], rr = bv[1], mid = bv[2];
    acc[0] = cadd(acc[0], cmul(mid, g_top[ky]));
    acc[1] = cadd(acc[1], cmul(mid, g_bot[ky]));
    acc[2] = cadd(acc[2], cmul(rl, g_kept[ky]));
    acc[3] = cadd(acc[3], cmul(rr, g_kept[ky]));
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int b = 0; b < 4; ++b) {
    acc[b] = lanes_sum<32>(acc[b]);
    if (lane == 0) part[warp][b] = acc[b];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const float s1 = (float)(1.0 / n), s2 = (float)(1.0 / ((double)n * n));
    for (int b = 0; b < 4; ++b) {
      float2 v = part[0][b];
      for (int q = 1; q < kWeightThreads / 32; ++q) v = cadd(v, part[q][b]);
      const float sc = b < 2 ? s1 : s2;
      sums[4 * t + b] = make_float2(v.x * sc, v.y * sc);
    }
    __threadfence();
    last = atomicAdd(counter, 1u) == (unsigned)ty - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  float2 *ss = chain_sm, *cs = chain_sm + 4 * ty;
  for (int q = threadIdx.x; q < 4 * ty; q += kWeightThreads) ss[q] = __ldcg(sums + 4 * ((q >> 2) * tx + j) + (q & 3));
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const float2 zero = make_float2(0.f, 0.f), one = make_float2(1.f, 0.f);
  // c(r) = c(r-1) B(r-1) / T(r), or 1 where T(r) = 0
  for (int r = lane; r < ty; r += 32) cs[r] = (r > 0 && cnonzero(ss[4 * r])) ? cdiv(ss[4 * (r - 1) + 1], ss[4 * r]) : one;
  __syncwarp();
  if (lane == 0) {
    float2 c = one;
    for (int r = 1; r < ty; ++r) {
      c = cnonzero(ss[4 * r]) ? cmul(c, cs[r]) : one;
      cs[r] = c;
    }
  }
  __syncwarp();
  float2 sl = zero, sr = zero;
  for (int r = lane; r < ty; r += 32) {
    sl = cadd(sl, cmul(cs[r], ss[4 * r + 2]));
    sr = cadd(sr, cmul(cs[r], ss[4 * r + 3]));
  }
  sl = lanes_sum<32>(sl);
  sr = lanes_sum<32>(sr);
  float2 d = one;
  if (j > 0 && cnonzero(sl)) d = cdiv(cmul(colst[0], colst[1]), sl);   // every lane: the same operands
  __syncwarp();
  if (lane == 0) {
    colst[0] = d;
    colst[1] = sr;
  }
  for (int r = lane; r < ty; r += 32) w[r * tx + j] = cmul(cs[r], d);
  if (lane == 0) *counter = 0u;
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
  const int T = p->n_tiles, n = g.n;
  const size_t nn = (size_t)n * n, fov = (size_t)g.fov_h * g.fov_w;
  // one tile column at a time: its row transforms (8 B per sample) wait in a
  // buffer of one tile column until its weights are known; two buffers, so that
  // the next column's row transforms run while this column's weights and
  // column transforms do (on the plan's second stream)
  Carve cv;
  const size_t o_buf = cv.take<float2>((size_t)2 * g.ty * nn), o_band = cv.take<float2>((size_t)2 * 3 * g.ty * n);
  const size_t o_sums = cv.take<float2>((size_t)4 * T), o_col = cv.take<float2>(2);
  const size_t o_cnt = cv.take<unsigned>(1), o_w = cv.take<float2>(T);
  const size_t o_out = on_device ? 0 : cv.take<float2>(fov);
  void *base = nullptr;
  if ((rc = fpm::plan_scratch(p, cv.off, &base))) return rc;
  char *b = static_cast<char *>(base);
  auto at = [&](size_t off) { return reinterpret_cast<float2 *>(b + off); };
  float2 *buf2[2] = {at(o_buf), at(o_buf) + (size_t)g.ty * nn};
  float2 *band2[2] = {at(o_band), at(o_band) + (size_t)3 * g.ty * n};
  float2 *sums = at(o_sums), *w = at(o_w);
  float2 *colst = at(o_col);
  unsigned *counter = reinterpret_cast<unsigned *>(b + o_cnt);
  float2 *out = on_device ? static_cast<float2 *>(dst) : at(o_out);
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned), st) != cudaSuccess)
    return fail(FPM_ECUDA, "fpm_stitch: counter reset failed");
  // the plan's tables: twiddles, twiddles in pass order and the band series
  float2 **slot = fpm::plan_stitch_tables(p);
  if (!slot) return fail(FPM_ESTATE, "fpm_stitch: no device state");
  if (!*slot) {
    const std::vector<float2> tab = fpm::stitch_tables(n, g.ov);
    if (cudaMalloc((void **)slot, tab.size() * sizeof(float2)) != cudaSuccess) {
      *slot = nullptr;
      return fail(FPM_ENOMEM, "fpm_stitch: table allocation failed");
    }
    if (cudaMemcpy(*slot, tab.data(), tab.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(FPM_ECUDA, "fpm_stitch: table upload failed");
  }
  const float2 *tw = *slot, *tw_pass = (n == 256 || n == 1024) ? *slot + n : nullptr;
  const float2 *gt = *slot + n + fpm::kPassTab;
  // the weights chain stages a tile column's sums and c values in shared memory
  const size_t chain_smem = (size_t)g.ty * 5 * sizeof(float2);
  if (chain_smem > 200 * 1024) return fail(FPM_EINVAL, "fpm_stitch: %d tile rows exceed the weight chain's limit", g.ty);
  if (chain_smem > 48 * 1024 &&
      cudaFuncSetAttribute((const void *)fpm::stitch_weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)chain_smem) != cudaSuccess)
    return fail(FPM_ECUDA, "fpm_stitch: weight kernel set-up failed");
  // per tile column j: 1. (stream st) row transforms of its spectra into buffer
  // j mod 2, with each row's band values; 2. (second stream) its band sums and
  // weights (Eq. 1 chained down the column and from column j - 1); 3. (second
  // stream) column transforms writing weight x (-1)^(x+y) / N^2 x result into the
  // image where the tile keeps the pixel.  Events order 2 after 1 and the row
  // transforms of column j + 2 after the column transforms of column j (same
  // buffer); the second stream starts after and ends before st's work.
  cudaStream_t aux = nullptr;
  cudaEvent_t *ev = nullptr;   // [0] fork, [1 + b] rows done in buffer b, [3 + b] buffer b free
  if ((rc = fpm::plan_stitch_streams(p, &aux, &ev))) return rc;
  auto ck = [&](cudaError_t e, const char *what) { return e == cudaSuccess ? FPM_OK : fail(FPM_ECUDA, "fpm_stitch: %s", what); };
  if ((rc = ck(cudaEventRecord(ev[0], st), "fork")) || (rc = ck(cudaStreamWaitEvent(aux, ev[0], 0), "fork")))
    return rc;
  const float scale = (float)(1.0 / ((double)n * n));
  for (int j = 0; j < g.tx; ++j) {
    const int bsel = j & 1;
    if (j >= 2 && (rc = ck(cudaStreamWaitEvent(st, ev[3 + bsel], 0), "buffer wait"))) return rc;
    if ((rc = fpm::launch_fft_rows_banded(buf2[bsel], fpm::plan_spectra(p) + (size_t)j * nn, tw, tw_pass, n, +1,
                                          g.ty, (long long)g.tx * nn, band2[bsel], g.ov, st)))
      return rc;
    if ((rc = ck(cudaEventRecord(ev[1 + bsel], st), "rows event")) ||
        (rc = ck(cudaStreamWaitEvent(aux, ev[1 + bsel], 0), "rows wait")))
      return rc;
    fpm::stitch_weights_kernel<<<(unsigned)g.ty, fpm::kWeightThreads, chain_smem, aux>>>(band2[bsel], gt, n, g.ty,
                                                                                        g.tx, j, sums, colst, counter, w);
    if (cudaGetLastError() != cudaSuccess) return fail(FPM_ECUDA, "fpm_stitch: weight kernel failed to launch");
    if ((rc = fpm::launch_fft_columns_to_fov(buf2[bsel], tw, tw_pass, n, +1, g.ty, scale, out, w, g.fov_w, g.ov, g.ty,
                                             g.tx, j, g.tx, aux)))
      return rc;
    if ((rc = ck(cudaEventRecord(ev[3 + bsel], aux), "columns event"))) return rc;
  }
  // join: st continues after the last column transforms
  if ((rc = ck(cudaStreamWaitEvent(st, ev[3 + ((g.tx - 1) & 1)], 0), "join"))) return rc;
  if (!on_device && cudaMemcpyAsync(dst, out, fov * sizeof(float2), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail(FPM_ECUDA, "fpm_stitch: copy out failed");
  return on_device ? FPM_OK : fpm::check_device_error(p, st);
}

}  // extern "C"
