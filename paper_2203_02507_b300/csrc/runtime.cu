// Host runtime of libfpm: device state of a plan, the initial guess, the
// reconstruction launch orchestration (plain, wave-batched, CUDA graph), the
// state getters/setters and the forward-model simulator.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "aux_kernels.cuh"
#include "internal.h"
#include "persistent.h"
#include "runtime.h"
#include "update.cuh"

namespace fpm {

#define FPM_CK(call)                                                                         \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(FPM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------------------------
// Update-kernel variants (tile side -> factorisation, cluster, threads)
// ---------------------------------------------------------------------------

using UpdateKernel = void (*)(UpdateArgs, long long);

struct Variant {
  int m, a, b, tpt, c, t;
  UpdateKernel k_u16, k_f32;
  size_t (*smem)(int rows);
  // the same variant with band pruning (UpdateCfg ZB = zb > 0), run where the
  // plan's support fits the band; null where the variant has none
  int zb = 0;
  UpdateKernel kz_u16 = nullptr, kz_f32 = nullptr;
};

template <class Cfg>
static Variant make_variant() {
  return Variant{Cfg::M, Cfg::A, Cfg::B, Cfg::TPT, Cfg::C, Cfg::T, &update_kernel<Cfg, uint16_t>,
                 &update_kernel<Cfg, float>, &Cfg::smem_bytes};
}

// A variant with a band-pruned twin: ZB blocks of B samples at each end of the
// box lie outside every support that the twin is run for.
template <class Cfg, int Z>
static Variant make_variant_band() {
  Variant v = make_variant<Cfg>();
  v.zb = Z;
  v.kz_u16 = &update_kernel<WithBand<Cfg, Z>, uint16_t>;
  v.kz_f32 = &update_kernel<WithBand<Cfg, Z>, float>;
  return v;
}

// The kernel of variant v for images of dtype: the band-pruned twin where the
// plan's support fits its band.
static UpdateKernel variant_kernel(const Variant *v, int dtype, bool band_ok) {
  if (v->zb > 0 && band_ok) return dtype == FPM_U16 ? v->kz_u16 : v->kz_f32;
  return dtype == FPM_U16 ? v->k_u16 : v->k_f32;
}

// Whether the plan's support lies in the band of the band-pruned update kernels
// (computed with the plan's support, fpm_plan_info.band).
bool plan_band_fits(const fpm_plan *p) { return p->band_ok; }

// candidates per tile side, preferred first; (m, A, B, lanes per transform, cluster, threads, min CTAs/SM)
using Cfg64 = UpdateCfg<64, 8, 8, 8, 1, 128, 4, 1, 0, 1>;
using Cfg64w = UpdateCfg<64, 8, 8, 8, 1, 256, 2>;
using Cfg64c2 = UpdateCfg<64, 8, 8, 8, 2, 128, 4, 1, 1>;
using Cfg64c4 = UpdateCfg<64, 8, 8, 8, 4, 128, 4, 1, 1, 1>;
using Cfg128 = UpdateCfg<128, 16, 8, 8, 1, 128, 2>;
using Cfg128w = UpdateCfg<128, 16, 8, 8, 1, 256, 1>;
using Cfg128o = UpdateCfg<128, 16, 8, 8, 2, 256, 2, 1, 0, 1>;
using Cfg128t = UpdateCfg<128, 16, 8, 8, 2, 128, 3, 1, 1, 1>;
using Cfg192 = UpdateCfg<192, 12, 16, 16, 1, 256, 1>;
using Cfg192c = UpdateCfg<192, 12, 16, 16, 2, 256, 1>;
using Cfg192h = UpdateCfg<192, 12, 16, 16, 2, 192, 2, 1, 1, 1>;
using Cfg192o = UpdateCfg<192, 12, 16, 16, 4, 256, 2, 1, 0, 1>;
using Cfg256 = UpdateCfg<256, 16, 16, 16, 2, 256, 1>;
using Cfg256w = UpdateCfg<256, 16, 16, 16, 2, 384, 1>;
using Cfg256x = UpdateCfg<256, 16, 16, 16, 2, 448, 1>;
using Cfg256q = UpdateCfg<256, 16, 16, 16, 4, 192, 2, 1, 1>;
using Cfg256o = UpdateCfg<256, 16, 16, 16, 4, 256, 2, 1, 0, 1>;
// eight lanes per transform (two radix units per lane and pass): the autotuner's
// threads-per-transform choice
using Cfg256e = UpdateCfg<256, 16, 16, 8, 4, 128, 2, 1, 0, 1>;
using Cfg128e = UpdateCfg<128, 16, 8, 4, 2, 128, 2, 1, 0, 1>;
using Cfg64e = UpdateCfg<64, 8, 8, 4, 1, 128, 2>;

static const std::vector<Variant> &variants() {
  static const std::vector<Variant> v = {
      make_variant<Cfg64>(),   make_variant<Cfg64w>(),  make_variant<Cfg64c2>(), make_variant<Cfg64c4>(),  // 64
      make_variant<Cfg64e>(),
      make_variant_band<Cfg128o, kBandBlocks>(), make_variant_band<Cfg128t, kBandBlocks>(), make_variant<Cfg128>(),
      make_variant<Cfg128w>(),                                                                           // 128
      make_variant<Cfg128e>(),
      make_variant<Cfg192h>(), make_variant<Cfg192o>(), make_variant<Cfg192>(),  make_variant<Cfg192c>(),  // 192
      make_variant_band<Cfg256o, kBandBlocks>(), make_variant<Cfg256x>(), make_variant<Cfg256q>(),
      make_variant<Cfg256w>(),
      make_variant<Cfg256>(),  make_variant<Cfg256e>()};                                                // 256
  return v;
}

static constexpr size_t kMaxSmem = 232448;   // 227 KB per CTA on sm_103a

// First candidate for tile side m whose shared memory fits; FPM_UPDATE_THREADS
// (environment) restricts the choice to one thread count ("448") or to one
// thread count and cluster size ("256x4").
static const Variant *find_variant(int m, int rows) {
  const char *env = getenv("FPM_UPDATE_THREADS");
  int want = 0, want_c = 0, want_l = 0;
  if (env && sscanf(env, "%dx%d/%d", &want, &want_c, &want_l) < 1) want = 0;
  for (const auto &v : variants())
    if (v.m == m && v.smem(rows) <= kMaxSmem && (want == 0 || v.t == want) && (want_c == 0 || v.c == want_c) &&
        (want_l == 0 || v.tpt == want_l))
      return &v;
  for (const auto &v : variants())
    if (v.m == m && v.smem(rows) <= kMaxSmem) return &v;
  return nullptr;
}

bool update_variant(int m, int rows, int *a, int *b, int *cluster, int *threads) {
  const Variant *v = find_variant(m, rows);
  if (!v) return false;
  *a = v->a;
  *b = v->b;
  *cluster = v->c;
  *threads = v->t;
  return true;
}

bool choose_launch(int32_t m, int32_t rows, int32_t *cluster, int32_t *threads) {
  const Variant *v = find_variant(m, rows);
  if (!v) return false;
  *cluster = v->c;
  *threads = v->t;
  return true;
}

// ---------------------------------------------------------------------------
// Twiddle tables (FP64 -> float)
// ---------------------------------------------------------------------------

void update_twiddles(int m, int a, int b, float2 *inv, float2 *fwd) {
  // inv[k1*B + b] = exp(+2 pi i b k1 / m), k1 < A, b < B
  // fwd[k1*A + b] = exp(-2 pi i b k1 / m), k1 < B, b < A
  for (int k1 = 0; k1 < a; ++k1)
    for (int bb = 0; bb < b; ++bb) {
      const double ang = 2.0 * M_PI * (double)(bb * k1) / m;
      inv[k1 * b + bb] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
  for (int k1 = 0; k1 < b; ++k1)
    for (int bb = 0; bb < a; ++bb) {
      const double ang = -2.0 * M_PI * (double)(bb * k1) / m;
      fwd[k1 * a + bb] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
}

std::vector<float2> twiddles_line(int len, int sign) {
  std::vector<float2> t(len);
  for (int j = 0; j < len; ++j) {
    const double ang = sign * 2.0 * M_PI * (double)j / len;
    t[j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  return t;
}

// Radix plan of a line FFT: 16s first, then 8, 4, 2 and a 3 (lengths 2^a or 3 * 2^a).
static bool radices_for(int len, FftLines &f) {
  int r = len, k = 0;
  if (r % 3 == 0) {
    f.radix[k++] = 3;
    r /= 3;
  }
  for (int rad : {16, 8, 4, 2})
    while (r % rad == 0 && k < kMaxRadices) {
      f.radix[k++] = rad;
      r /= rad;
    }
  f.nrad = k;
  return r == 1 && len <= kMaxFftLen;
}

// ---------------------------------------------------------------------------
// Device state
// ---------------------------------------------------------------------------

struct DeviceBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

struct StepDev {
  int32_t iters = 0;
  int4 *items = nullptr;
  int2 *merges = nullptr;         // (tile, slots) per step, see StepLists
};

struct GraphKey {
  int32_t iters, mode;
  cudaStream_t stream;
  bool operator<(const GraphKey &o) const {
    return iters != o.iters ? iters < o.iters : mode != o.mode ? mode < o.mode : stream < o.stream;
  }
};

constexpr int kMaxBranches = 8;

struct DeviceState {
  int device = -1;
  float2 *spec = nullptr, *pup = nullptr, *dpup = nullptr;   // pup: [T][m][m]; dpup: [T][W][m][m]
  float2 *pup0 = nullptr;                           // initial pupils [T][m][m] (each load starts from them)
  int2 *shifts = nullptr, *origins = nullptr, *chords = nullptr;
  float2 *tw_inv = nullptr, *tw_fwd = nullptr;      // update kernel split
  float2 *twl_fwd_m = nullptr;                      // line FFT tables
  float2 *stitch_tab = nullptr;                     // tables of the stitch (built on its first call)

  unsigned *err = nullptr;
  void *images = nullptr;                          // [T][L][m][m] column layout (tile_image_offset)
  size_t images_bytes = 0;
  void *scratch = nullptr;                         // temporaries of the object / stitch calls
  size_t scratch_bytes = 0;
  int32_t dtype = FPM_U16;
  float inv_counts = 1.f;
  bool loaded = false;
  const Variant *var = nullptr;
  bool band_ok = false;                            // the support fits the band-pruned kernels' band
  std::vector<StepDev> steps;
  std::map<GraphKey, cudaGraphExec_t> graphs;
  std::map<GraphKey, int64_t> graph_launches;
  std::map<GraphKey, int32_t> graph_threads;      // update-kernel threads captured in each graph
  int32_t run_threads = 0;                        // of the last fpm_reconstruct (fpm_get_stats)
  int32_t run_cluster = 0;
  int32_t run_lanes = 0;
  std::map<GraphKey, int32_t> graph_cluster;      // its CTAs per cluster
  std::map<GraphKey, int32_t> graph_lanes;        // its lanes per transform
  // counters (fpm_get_stats)
  int64_t load_launches = 0, run_launches = 0;
  std::vector<cudaEvent_t> events;            // 2 per wave step of a timed run
  std::vector<int64_t> timed_steps;           // steps whose update launch was timed
  int64_t timed_n_steps = 0;                  // steps of the timed schedule (its closing event)
  int64_t timed_updates = 0;
  bool timed_valid = false;
  std::map<int32_t, QueueDev *> queues;        // persistent queues by loop count
  int persistent_clusters = 0;
  int tuned_mode = FPM_RUN_PERSISTENT;         // FPM_RUN_AUTO resolves to this
  // graph replays of FPM_RUN_WAVES split the tiles into `branches` groups whose
  // wave steps run as parallel branches of the graph (tiles are independent)
  int32_t branches = 1;
  cudaStream_t branch_st[kMaxBranches] = {};
  cudaEvent_t branch_ev[2 * kMaxBranches] = {};
  cudaStream_t batch_st = nullptr;                 // this plan's part of a wave-mode batch
  cudaEvent_t batch_ev[2] = {};
  cudaStream_t stitch_st = nullptr;                // the stitch's second stream and its events
  cudaEvent_t stitch_ev[kStitchEvents] = {};
};

static void dfree(void *p) {
  if (p) cudaFree(p);
}

void forget_batches(fpm_plan *p);

void destroy_device_state(fpm_plan *p) {
  destroy_online_state(p);
  DeviceState *d = p->dev;
  if (!d) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (d->device >= 0) cudaSetDevice(d->device);
  cudaDeviceSynchronize();
  for (auto &kv : d->graphs) cudaGraphExecDestroy(kv.second);
  for (cudaEvent_t ev : d->events) cudaEventDestroy(ev);
  for (cudaStream_t bs : d->branch_st)
    if (bs) cudaStreamDestroy(bs);
  for (cudaEvent_t ev : d->branch_ev)
    if (ev) cudaEventDestroy(ev);
  if (d->batch_st) cudaStreamDestroy(d->batch_st);
  for (cudaEvent_t ev : d->batch_ev)
    if (ev) cudaEventDestroy(ev);
  if (d->stitch_st) cudaStreamDestroy(d->stitch_st);
  for (cudaEvent_t ev : d->stitch_ev)
    if (ev) cudaEventDestroy(ev);
  for (auto &kv : d->queues) free_queue(kv.second);
  forget_batches(p);
  for (auto &s : d->steps) {
    dfree(s.items);
    dfree(s.merges);
  }
  for (void *q : {(void *)d->spec, (void *)d->pup, (void *)d->pup0, (void *)d->dpup, (void *)d->shifts, (void *)d->origins,
                  (void *)d->chords, (void *)d->tw_inv, (void *)d->tw_fwd, (void *)d->twl_fwd_m, (void *)d->stitch_tab, (void *)d->err,
                  d->images, d->scratch})
    dfree(q);
  if (cur >= 0) cudaSetDevice(cur);
  delete d;
  p->dev = nullptr;
}

template <class T>
static int upload(T **dst, const void *src, size_t bytes) {
  FPM_CK(cudaMalloc((void **)dst, bytes));
  FPM_CK(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
  return FPM_OK;
}

int ensure_device_state(fpm_plan *p) {
  if (p->dev) return FPM_OK;
  DeviceState *d = new DeviceState();
  p->dev = d;
  FPM_CK(cudaGetDevice(&d->device));
  const int rows = p->y_hi - p->y_lo + 1;
  d->var = find_variant(p->m, rows);
  if (!d->var) return fail(FPM_EINVAL, "no update kernel for tile %d with %d support rows", p->m, rows);
  d->band_ok = plan_band_fits(p);
  if (const char *env = getenv("FPM_WAVE_BRANCHES")) d->branches = std::max(1, std::min(kMaxBranches, atoi(env)));
  if (!persistent_fits(p->m, rows)) d->tuned_mode = FPM_RUN_WAVES;   // FPM_RUN_AUTO before any tuning
  const size_t T = p->n_tiles, n = p->n, m = p->m;
  cudaError_t e;
  for (const auto &v : variants())            // every fitting variant may be chosen by the autotuner
    if (v.m == p->m && v.smem(rows) <= kMaxSmem) {
      FPM_CK(cudaFuncSetAttribute((const void *)v.k_u16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)v.smem(rows)));
      FPM_CK(cudaFuncSetAttribute((const void *)v.k_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)v.smem(rows)));
      if (v.zb > 0) {
        FPM_CK(cudaFuncSetAttribute((const void *)v.kz_u16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)v.smem(rows)));
        FPM_CK(cudaFuncSetAttribute((const void *)v.kz_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)v.smem(rows)));
      }
    }
  if ((e = cudaMalloc((void **)&d->spec, T * n * n * sizeof(float2))) != cudaSuccess ||
      (e = cudaMalloc((void **)&d->pup, T * m * m * sizeof(float2))) != cudaSuccess)
    return fail(FPM_ENOMEM, "device allocation of the tile state failed: %s", cudaGetErrorString(e));
  if ((e = cudaMalloc((void **)&d->pup0, T * m * m * sizeof(float2))) != cudaSuccess)
    return fail(FPM_ENOMEM, "device allocation of the initial pupils failed: %s", cudaGetErrorString(e));
  FPM_CK(cudaMemcpy(d->pup0, p->pupil0.data(), T * m * m * sizeof(float2), cudaMemcpyHostToDevice));
  if (p->epry) {
    const size_t db = T * (size_t)p->max_width * m * m * sizeof(float2);
    if ((e = cudaMalloc((void **)&d->dpup, db)) != cudaSuccess)
      return fail(FPM_ENOMEM, "device allocation of the pupil corrections failed: %s", cudaGetErrorString(e));
    FPM_CK(cudaMemset(d->dpup, 0, db));   // the merge sums whole pixel pairs: off-support entries stay zero
  }
  std::vector<int2> sh((size_t)p->n_tiles * p->n_leds), org(p->n_tiles), ch(p->m);
  for (size_t i = 0; i < sh.size(); ++i) sh[i] = make_int2(p->shifts[i * 2], p->shifts[i * 2 + 1]);
  for (int t = 0; t < p->n_tiles; ++t) {
    org[t] = make_int2(p->origins[t * 2], p->origins[t * 2 + 1]);
  }
  for (int i = 0; i < p->m; ++i) ch[i] = make_int2(p->chord_lo[i], p->chord_hi[i]);
  int rc;
  if ((rc = upload(&d->shifts, sh.data(), sh.size() * sizeof(int2)))) return rc;
  if ((rc = upload(&d->origins, org.data(), org.size() * sizeof(int2)))) return rc;
  if ((rc = upload(&d->chords, ch.data(), ch.size() * sizeof(int2)))) return rc;
  std::vector<float2> ti(p->m), tf(p->m);
  update_twiddles(p->m, d->var->a, d->var->b, ti.data(), tf.data());
  if ((rc = upload(&d->tw_inv, ti.data(), ti.size() * sizeof(float2)))) return rc;
  if ((rc = upload(&d->tw_fwd, tf.data(), tf.size() * sizeof(float2)))) return rc;
  std::vector<float2> tl = twiddles_line(p->m, -1);
  if ((rc = upload(&d->twl_fwd_m, tl.data(), tl.size() * sizeof(float2)))) return rc;
  FPM_CK(cudaMalloc((void **)&d->err, 4 * sizeof(unsigned)));
  FPM_CK(cudaMemset(d->err, 0, 4 * sizeof(unsigned)));
  const size_t smem = d->var->smem(rows);
  FPM_CK(cudaFuncSetAttribute((const void *)variant_kernel(d->var, FPM_U16, d->band_ok),
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FPM_CK(cudaFuncSetAttribute((const void *)variant_kernel(d->var, FPM_F32, d->band_ok),
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return FPM_OK;
}

// Batched 1-D FFTs over lines of a device array.
// Launch the line transforms described by f (data, src, tw, len, strides, lines
// per batch, finish and the optional field-of-view output already set).
static int launch_lines(FftLines f, int sign, long long n_lines, cudaStream_t st) {
  const int len = f.len;
  if (f.src_batch_stride == 0) f.src_batch_stride = f.batch_stride;
  if (f.fov_tile_step == 0) f.fov_tile_step = 1;
  const long long lines_per_batch = f.lines_per_batch, batch_stride = f.batch_stride;
  const long long src_batch_stride = f.src_batch_stride;
  float2 *const data = f.data;
  const float2 *const src = f.src;
  float2 *const band = f.band;
  const int tile0 = f.fov_tile0;
  if (!radices_for(len, f)) return fail(FPM_EINVAL, "FFT length %d not supported", len);
  if (band && f.elem_stride != 1) return fail(FPM_EINVAL, "internal: band sums need contiguous lines");
  // lengths 256 and 1024: butterflies in registers, G lines per CTA (rows: any lines;
  // strided samples: G adjacent lines of one batch)
  if (len == 256 || len == 1024) {
    const bool rows = f.elem_stride == 1;
    // strided 1024-sample lines: 8 adjacent ones per CTA, 64-byte row segments
    const int G = len == 256 ? 16 : rows ? 4 : 8;
    const bool cols = f.line_stride == 1 && lines_per_batch % G == 0;
    if ((rows || cols) && n_lines % G == 0 && !(rows && f.fov)) {
      void (*kern)(FftLines);
      const bool tp = f.tw_pass != nullptr;
      if (len == 256)
        kern = tp ? (sign > 0 ? &fft_lines_reg_kernel<1, 256, 16, true> : &fft_lines_reg_kernel<-1, 256, 16, true>)
                  : (sign > 0 ? &fft_lines_reg_kernel<1, 256, 16, false> : &fft_lines_reg_kernel<-1, 256, 16, false>);
      else if (rows)
        kern = tp ? (sign > 0 ? &fft_lines_reg_kernel<1, 1024, 4, true> : &fft_lines_reg_kernel<-1, 1024, 4, true>)
                  : (sign > 0 ? &fft_lines_reg_kernel<1, 1024, 4, false> : &fft_lines_reg_kernel<-1, 1024, 4, false>);
      else
        kern = tp ? (sign > 0 ? &fft_lines_reg_kernel<1, 1024, 8, true> : &fft_lines_reg_kernel<-1, 1024, 8, true>)
                  : (sign > 0 ? &fft_lines_reg_kernel<1, 1024, 8, false> : &fft_lines_reg_kernel<-1, 1024, 8, false>);
      const size_t smem = (size_t)G * line_padded_len(len, G) * sizeof(float2);
      FPM_CK(cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      const long long max_chunk = (1LL << 30) / lines_per_batch * lines_per_batch;   // whole batches per launch
      for (long long done = 0; done < n_lines;) {
        const long long chunk = std::min<long long>(n_lines - done, max_chunk);
        FftLines g = f;
        const long long bdone = done / lines_per_batch;
        g.data = data + bdone * batch_stride;
        g.src = src ? src + bdone * src_batch_stride : nullptr;
        g.band = band ? band + 3 * done : nullptr;
        g.fov_tile0 = tile0 + (int)bdone * f.fov_tile_step;
        kern<<<(unsigned)(chunk / G), G * (len / 16), smem, st>>>(g);
        done += chunk;
      }
      FPM_CK(cudaGetLastError());
      return FPM_OK;
    }
  }
  if (f.fov && f.elem_stride == 1) return fail(FPM_EINVAL, "internal: field-of-view output needs strided lines");
  // strided lines (columns): four adjacent ones per CTA, so loads and stores use whole sectors
  f.lines_per_cta =
      (f.line_stride == 1 && f.elem_stride > 1 && lines_per_batch % 4 == 0 && n_lines % 4 == 0) ? 4 : 1;
  // one group of threads per line, a thread per radix-16 butterfly (whole warps)
  const int group = std::min(256, std::max(32, (len / 16 + 31) / 32 * 32));
  const int threads = group * f.lines_per_cta;
  const size_t smem = (size_t)f.lines_per_cta * 2 * line_padded_len(len) * sizeof(float2);
  void (*kern)(FftLines);
  if (f.lines_per_cta == 4) kern = sign > 0 ? &fft_lines_kernel<1, 4> : &fft_lines_kernel<-1, 4>;
  else kern = sign > 0 ? &fft_lines_kernel<1, 1> : &fft_lines_kernel<-1, 1>;
  FPM_CK(cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const long long max_chunk = (1LL << 30) / lines_per_batch * lines_per_batch;   // whole batches per launch
  for (long long done = 0; done < n_lines;) {
    const long long chunk = std::min<long long>(n_lines - done, max_chunk);
    FftLines g = f;
    // offset the bases so that line indices restart at a batch boundary
    const long long first = done;
    if (first % lines_per_batch != 0) return fail(FPM_EINVAL, "internal: FFT chunk not batch aligned");
    const long long bdone = first / lines_per_batch;
    g.data = data + bdone * batch_stride;
    g.src = src ? src + bdone * src_batch_stride : nullptr;
    g.band = band ? band + 3 * first : nullptr;
    g.fov_tile0 = tile0 + (int)bdone * f.fov_tile_step;
    const unsigned ctas = (unsigned)(chunk / f.lines_per_cta);
    kern<<<ctas, threads, smem, st>>>(g);
    done += chunk;
  }
  FPM_CK(cudaGetLastError());
  return FPM_OK;
}

int launch_fft_lines_ex(float2 *data, const float2 *src, const float2 *tw, int len, int sign, long long n_lines,
                        int lines_per_batch, long long batch_stride, long long line_stride, long long elem_stride,
                        float finish, cudaStream_t st) {
  FftLines f{};
  f.data = data;
  f.src = src;
  f.tw = tw;
  f.len = len;
  f.batch_stride = batch_stride;
  f.line_stride = line_stride;
  f.elem_stride = elem_stride;
  f.lines_per_batch = lines_per_batch;
  f.finish = finish;
  return launch_lines(f, sign, n_lines, st);
}

int launch_fft_rows_banded(float2 *data, const float2 *src, const float2 *tw, const float2 *tw_pass, int n, int sign,
                           int tiles, long long src_tile_stride, float2 *band, int ov, cudaStream_t st) {
  FftLines f{};
  f.data = data;
  f.src = src;
  f.tw = tw;
  f.tw_pass = tw_pass;
  f.len = n;
  f.batch_stride = (long long)n * n;
  f.src_batch_stride = src_tile_stride;
  f.line_stride = n;
  f.elem_stride = 1;
  f.lines_per_batch = n;
  f.band = band;
  f.band_ov = ov;
  return launch_lines(f, sign, (long long)tiles * n, st);
}

int launch_fft_columns_to_fov(const float2 *data, const float2 *tw, const float2 *tw_pass, int n, int sign, int tiles,
                              float finish, float2 *fov, const float2 *weight, long long fov_w, int ov, int tiles_y,
                              int tiles_x, int tile0, int tile_step, cudaStream_t st) {
  FftLines f{};
  f.data = const_cast<float2 *>(data);      // read only: the output goes to fov
  f.src = nullptr;
  f.tw = tw;
  f.tw_pass = tw_pass;
  f.len = n;
  f.batch_stride = (long long)n * n;
  f.line_stride = 1;
  f.elem_stride = n;
  f.lines_per_batch = n;
  f.finish = finish;
  f.fov = fov;
  f.fov_weight = weight;
  f.fov_w = fov_w;
  f.fov_ov = ov;
  f.fov_tiles_y = tiles_y;
  f.fov_tiles_x = tiles_x;
  f.fov_tile0 = tile0;
  f.fov_tile_step = tile_step;
  return launch_lines(f, sign, (long long)tiles * n, st);
}

int launch_fft_lines(float2 *data, const float2 *tw, int len, int sign, long long n_lines, int lines_per_batch,
                     long long batch_stride, long long line_stride, long long elem_stride, cudaStream_t st) {
  return launch_fft_lines_ex(data, nullptr, tw, len, sign, n_lines, lines_per_batch, batch_stride, line_stride,
                             elem_stride, 0.f, st);
}

static unsigned grid_for(long long n, int threads) {
  return (unsigned)std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, 148LL * 64));
}

// Initial guess of every tile from its image of the first LED in the order.
// `plane` is the sensor image of the first LED of the order (rows stride_row
// elements apart).
int run_init(fpm_plan *p, const void *plane, long long stride_row, cudaStream_t st) {
  DeviceState *d = p->dev;
  const int m = p->m, n = p->n, T = p->n_tiles;
  float2 *tmp = nullptr;
  FPM_CK(cudaMallocAsync((void **)&tmp, (size_t)T * m * m * sizeof(float2), st));
  const long long tot = (long long)T * m * m;
  const void *stack = plane;
  const long long stride_led = 0;
  const int led = 0;
  if (d->dtype == FPM_U16)
    init_gather_kernel<uint16_t><<<grid_for(tot, 256), 256, 0, st>>>(
        tmp, (const uint16_t *)stack, stride_led, stride_row, d->origins, led, m, T, d->inv_counts);
  else
    init_gather_kernel<float><<<grid_for(tot, 256), 256, 0, st>>>(tmp, (const float *)stack, stride_led, stride_row,
                                                                    d->origins, led, m, T, d->inv_counts);
  int rc;
  // rows then columns of every tile
  if ((rc = launch_fft_lines(tmp, d->twl_fwd_m, m, -1, (long long)T * m, m, (long long)m * m, m, 1, st))) return rc;
  if ((rc = launch_fft_lines(tmp, d->twl_fwd_m, m, -1, (long long)T * m, m, (long long)m * m, 1, m, st))) return rc;
  FPM_CK(cudaMemsetAsync(d->spec, 0, (size_t)T * n * n * sizeof(float2), st));
  const float scale = (float)((double)n / m * (double)n / m);
  init_place_kernel<<<grid_for(tot, 256), 256, 0, st>>>(d->spec, tmp, m, n, T, scale);
  FPM_CK(cudaGetLastError());
  FPM_CK(cudaFreeAsync(tmp, st));
  // pupils into buffer 0
  FPM_CK(cudaMemcpyAsync(d->pup, d->pup0, (size_t)T * m * m * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  d->load_launches = 5;   // tile images, gather, 2 x line FFT, place
  return FPM_OK;
}

static const StepDev *device_steps(fpm_plan *p, int32_t iters, const StepLists &sl, int *rc) {
  DeviceState *d = p->dev;
  for (auto &s : d->steps)
    if (s.iters == iters) return &s;
  StepDev s;
  s.iters = iters;
  *rc = upload(&s.items, sl.items.data(), std::max<size_t>(sl.items.size(), 4) * sizeof(int32_t));
  if (*rc) return nullptr;
  *rc = upload(&s.merges, sl.merges.data(), std::max<size_t>(sl.merges.size(), 2) * sizeof(int32_t));
  if (*rc) return nullptr;
  d->steps.push_back(s);
  return &d->steps.back();
}

static UpdateArgs make_args(fpm_plan *p, const StepDev *sd) {
  DeviceState *d = p->dev;
  UpdateArgs a{};
  a.spec = d->spec;
  a.pup = d->pup;
  a.dpup = p->epry ? d->dpup : nullptr;
  a.items = sd ? sd->items : nullptr;
  a.shifts = d->shifts;
  a.chords = d->chords;
  a.tw_inv = d->tw_inv;
  a.tw_fwd = d->tw_fwd;
  a.images = d->images;
  a.inv_counts = d->inv_counts;
  a.scale = (float)((double)p->n / p->m * (double)p->n / p->m);
  a.n = p->n;
  a.n_leds = p->n_leds;
  a.y_lo = p->y_lo;
  a.rows = p->y_hi - p->y_lo + 1;
  a.slots = p->max_width;
  a.disc = p->disc_ok ? 1 : 0;
  a.err = d->err;
  return a;
}

static int launch_update(fpm_plan *p, const UpdateArgs &a, long long item0, long long count, cudaStream_t st) {
  if (count <= 0) return FPM_OK;
  DeviceState *d = p->dev;
  const Variant *v = d->var;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(count * v->c), 1, 1);
  cfg.blockDim = dim3(v->t, 1, 1);
  cfg.dynamicSmemBytes = v->smem(a.rows);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = v->c;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = v->c > 1 ? 1 : 0;
  UpdateKernel k = variant_kernel(v, d->dtype, d->band_ok);
  FPM_CK(cudaLaunchKernelEx(&cfg, k, a, item0));
  return FPM_OK;
}

int launch_update_items(int m, int rows, int dtype, const UpdateArgs &a, long long item0, long long count,
                        cudaStream_t st, bool band) {
  const Variant *v = find_variant(m, rows);
  if (!v) return fail(FPM_EINVAL, "no update kernel for tile %d with %d support rows", m, rows);
  if (count <= 0) return FPM_OK;
  const size_t smem = v->smem(rows);
  UpdateKernel k = variant_kernel(v, dtype, band);
  FPM_CK(cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(count * v->c), 1, 1);
  cfg.blockDim = dim3(v->t, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = v->c;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = v->c > 1 ? 1 : 0;
  FPM_CK(cudaLaunchKernelEx(&cfg, k, a, item0));
  return FPM_OK;
}

int launch_merge(float2 *pup, const float2 *dpup, const int2 *entries, int count, int y_lo, int rows, int m,
                 int slots, int disc, cudaStream_t st) {
  if (count <= 0) return FPM_OK;
  merge_kernel<<<dim3((unsigned)count, kNormParts), 256, 0, st>>>(pup, dpup, entries, y_lo, rows, m, slots, disc);
  FPM_CK(cudaGetLastError());
  return FPM_OK;
}

UpdateArgs plan_update_args(fpm_plan *p) { return make_args(p, nullptr); }

int plan_image_dtype(const fpm_plan *p) { return (p->dev && p->dev->loaded) ? p->dev->dtype : -1; }

unsigned *plan_error_word(fpm_plan *p) { return p->dev ? p->dev->err : nullptr; }

const float2 *plan_spectra(const fpm_plan *p) { return (p->dev && p->dev->loaded) ? p->dev->spec : nullptr; }
float2 **plan_stitch_tables(fpm_plan *p) { return p->dev ? &p->dev->stitch_tab : nullptr; }

int plan_stitch_streams(fpm_plan *p, cudaStream_t *aux, cudaEvent_t **ev) {
  DeviceState *d = p->dev;
  if (!d) return fail(FPM_ESTATE, "no device state before fpm_load_tiles");
  if (!d->stitch_st) {
    if (cudaStreamCreateWithFlags(&d->stitch_st, cudaStreamNonBlocking) != cudaSuccess) {
      d->stitch_st = nullptr;
      return fail(FPM_ECUDA, "stitch stream creation failed");
    }
    for (cudaEvent_t &e : d->stitch_ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        // undo, so that the next call tries again from scratch
        e = nullptr;
        for (cudaEvent_t &x : d->stitch_ev)
          if (x) cudaEventDestroy(x), x = nullptr;
        cudaStreamDestroy(d->stitch_st);
        d->stitch_st = nullptr;
        return fail(FPM_ECUDA, "stitch event creation failed");
      }
  }
  *aux = d->stitch_st;
  *ev = d->stitch_ev;
  return FPM_OK;
}

int plan_scratch(fpm_plan *p, size_t bytes, void **out) {
  DeviceState *d = p->dev;
  *out = nullptr;
  if (!d) return fail(FPM_ESTATE, "no device state before fpm_load_tiles");
  if (d->scratch_bytes < bytes) {
    if (d->scratch) cudaFree(d->scratch);          // synchronises: earlier users are done
    d->scratch = nullptr;
    d->scratch_bytes = 0;
    if (cudaMalloc(&d->scratch, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(FPM_ENOMEM, "device allocation of %zu bytes of scratch failed", bytes);
    }
    d->scratch_bytes = bytes;
  }
  *out = d->scratch;
  return FPM_OK;
}

// Enqueue the launches of `iters` loops in the given mode; *launches counts kernels.
// With `timed`, CUDA events bracket every update launch (waves mode only).
static int enqueue_wave_branches(fpm_plan *p, int32_t iters, int s0, int s1, int branches, cudaStream_t st,
                                 int64_t *launches);
static int enqueue_wave_tiles(fpm_plan *p, int32_t iters, int s0, int s1, int t0, int t1, cudaStream_t st,
                              int64_t *launches);

// Wave steps [s0, s1) captured as one graph of `branches` tile-group branches.
int capture_wave_steps(fpm_plan *p, int32_t iters, int s0, int s1, int branches, cudaGraphExec_t *out) {
  *out = nullptr;
  const StepLists &sl = step_lists(p, iters);
  int rc = 0;
  if (!device_steps(p, iters, sl, &rc)) return rc;            // uploads stay outside the capture
  cudaStream_t cap = nullptr;
  FPM_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  int64_t nl = 0;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const int b = std::min(branches, std::max(1, p->n_tiles));
    rc = b > 1 ? enqueue_wave_branches(p, iters, s0, s1, b, cap, &nl)
               : enqueue_wave_tiles(p, iters, s0, s1, 0, p->n_tiles, cap, &nl);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    if (!rc && e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
  }
  cudaStreamDestroy(cap);
  if (rc) return rc;
  if (e != cudaSuccess) return fail(FPM_ECUDA, "capture of wave steps: %s", cudaGetErrorString(e));
  return FPM_OK;
}

// Wave steps [s0, s1) of the `iters`-loop schedule, as FPM_RUN_WAVES runs them:
// each step's update launch, then (EPRY) its pupil merge; with the plan's
// branch count above 1, two tile groups' parts as parallel branches (launched
// one by one, not replayed as a graph: more branches make the host's launch
// rate the limit).
int enqueue_wave_steps(fpm_plan *p, int32_t iters, int s0, int s1, cudaStream_t st) {
  const int b = std::min(std::min(p->dev->branches, 2), std::max(1, p->n_tiles));
  if (b > 1) {
    int64_t nl = 0;
    return enqueue_wave_branches(p, iters, s0, s1, b, st, &nl);
  }
  const StepLists &sl = step_lists(p, iters);
  int rc = 0;
  const StepDev *sd = device_steps(p, iters, sl, &rc);
  if (!sd) return rc;
  const UpdateArgs a = make_args(p, sd);
  DeviceState *d = p->dev;
  const int rows = p->y_hi - p->y_lo + 1;
  for (int s = std::max(0, s0); s < std::min(s1, sl.n_steps); ++s) {
    const long long i0 = sl.step_off[s], i1 = sl.step_off[s + 1];
    if ((rc = launch_update(p, a, i0, i1 - i0, st))) return rc;
    if (p->epry) {
      const long long m0 = sl.merge_off[s], m1 = sl.merge_off[s + 1];
      if ((rc = launch_merge(d->pup, d->dpup, sd->merges + m0, (int)(m1 - m0), p->y_lo, rows, p->m, p->max_width,
                             p->disc_ok ? 1 : 0, st)))
        return rc;
    }
  }
  FPM_CK(cudaGetLastError());
  return FPM_OK;
}

// Wave steps [s0, s1) of the `iters`-loop schedule restricted to tiles [t0, t1)
// (a step's items and merges are sorted by tile, so the range is contiguous).
static int enqueue_wave_tiles(fpm_plan *p, int32_t iters, int s0, int s1, int t0, int t1, cudaStream_t st,
                              int64_t *launches) {
  const StepLists &sl = step_lists(p, iters);
  int rc = 0;
  const StepDev *sd = device_steps(p, iters, sl, &rc);
  if (!sd) return rc;
  const UpdateArgs a = make_args(p, sd);
  DeviceState *d = p->dev;
  const int rows = p->y_hi - p->y_lo + 1;
  const int32_t *items = sl.items.data(), *merges = sl.merges.data();
  auto first_item = [&](int64_t lo, int64_t hi, int t) {       // first item of tile >= t in [lo, hi)
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (items[mid * 4] < t) lo = mid + 1;
      else hi = mid;
    }
    return lo;
  };
  auto first_merge = [&](int64_t lo, int64_t hi, int t) {
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (merges[mid * 2] < t) lo = mid + 1;
      else hi = mid;
    }
    return lo;
  };
  int64_t nl = 0;
  for (int s = std::max(0, s0); s < std::min(s1, sl.n_steps); ++s) {
    const int64_t i0 = first_item(sl.step_off[s], sl.step_off[s + 1], t0);
    const int64_t i1 = first_item(i0, sl.step_off[s + 1], t1);
    if (i1 == i0) continue;
    if ((rc = launch_update(p, a, i0, i1 - i0, st))) return rc;
    ++nl;
    if (p->epry) {
      const int64_t m0 = first_merge(sl.merge_off[s], sl.merge_off[s + 1], t0);
      const int64_t m1 = first_merge(m0, sl.merge_off[s + 1], t1);
      if ((rc = launch_merge(d->pup, d->dpup, sd->merges + m0, (int)(m1 - m0), p->y_lo, rows, p->m, p->max_width,
                             p->disc_ok ? 1 : 0, st)))
        return rc;
      if (m1 > m0) ++nl;
    }
  }
  FPM_CK(cudaGetLastError());
  *launches += nl;
  return FPM_OK;
}

// Wave steps [s0, s1) as `branches` parallel branches over tile groups: forked
// from and joined back into the stream st (capturing or not) with events.
static int enqueue_wave_branches(fpm_plan *p, int32_t iters, int s0, int s1, int branches, cudaStream_t st,
                                 int64_t *launches) {
  DeviceState *d = p->dev;
  for (int k = 0; k < branches; ++k) {
    if (k > 0 && !d->branch_st[k]) FPM_CK(cudaStreamCreateWithFlags(&d->branch_st[k], cudaStreamNonBlocking));
    for (int e = 0; e < 2; ++e)
      if (!d->branch_ev[2 * k + e]) FPM_CK(cudaEventCreateWithFlags(&d->branch_ev[2 * k + e], cudaEventDisableTiming));
  }
  FPM_CK(cudaEventRecord(d->branch_ev[0], st));                 // fork
  for (int k = 1; k < branches; ++k) FPM_CK(cudaStreamWaitEvent(d->branch_st[k], d->branch_ev[0], 0));
  int rc = FPM_OK;
  for (int k = 0; k < branches && rc == FPM_OK; ++k) {
    const int t0 = (int)((int64_t)p->n_tiles * k / branches), t1 = (int)((int64_t)p->n_tiles * (k + 1) / branches);
    rc = enqueue_wave_tiles(p, iters, s0, s1, t0, t1, k == 0 ? st : d->branch_st[k], launches);
  }
  for (int k = 1; k < branches; ++k) {                          // join (also after a failure, to end the capture cleanly)
    FPM_CK(cudaEventRecord(d->branch_ev[2 * k + 1], d->branch_st[k]));
    FPM_CK(cudaStreamWaitEvent(st, d->branch_ev[2 * k + 1], 0));
  }
  return rc;
}

static int enqueue_reconstruct(fpm_plan *p, int32_t iters, int mode, cudaStream_t st, bool timed, bool capturing,
                               int64_t *launches) {
  const StepLists &sl = step_lists(p, iters);
  int rc = 0;
  const StepDev *sd = device_steps(p, iters, sl, &rc);
  if (!sd) return rc;
  const UpdateArgs a = make_args(p, sd);
  DeviceState *d = p->dev;
  const int rows = p->y_hi - p->y_lo + 1;
  int64_t nl = 0;
  if (mode == FPM_RUN_WAVES) {
    if (timed) {
      while ((int)d->events.size() < 2 * sl.n_steps + 1) {
        cudaEvent_t ev;
        FPM_CK(cudaEventCreate(&ev));
        d->events.push_back(ev);
      }
      d->timed_steps.clear();
      d->timed_updates = 0;
      d->timed_valid = true;
      d->timed_n_steps = sl.n_steps;
    }
    for (int s = 0; s < sl.n_steps; ++s) {
      const long long i0 = sl.step_off[s], i1 = sl.step_off[s + 1];
      if (timed && i1 > i0) {
        FPM_CK(capturing ? cudaEventRecordWithFlags(d->events[2 * s], st, cudaEventRecordExternal)
                         : cudaEventRecord(d->events[2 * s], st));
      }
      if ((rc = launch_update(p, a, i0, i1 - i0, st))) return rc;
      if (i1 > i0) ++nl;
      if (timed && i1 > i0) {
        FPM_CK(capturing ? cudaEventRecordWithFlags(d->events[2 * s + 1], st, cudaEventRecordExternal)
                         : cudaEventRecord(d->events[2 * s + 1], st));
        d->timed_steps.push_back(s);
        d->timed_updates += i1 - i0;
      }
      if (p->epry) {   // close the wave: its corrections into the pupils, in sequence order
        const long long m0 = sl.merge_off[s], m1 = sl.merge_off[s + 1];
        if ((rc = launch_merge(d->pup, d->dpup, sd->merges + m0, (int)(m1 - m0), p->y_lo, rows, p->m,
                               p->max_width, p->disc_ok ? 1 : 0, st)))
          return rc;
        if (m1 > m0) ++nl;
      }
    }
    if (timed)   // closes the last merge: merges run between an update's end and the next start
      FPM_CK(capturing ? cudaEventRecordWithFlags(d->events[2 * sl.n_steps], st, cudaEventRecordExternal)
                       : cudaEventRecord(d->events[2 * sl.n_steps], st));
    FPM_CK(cudaGetLastError());
    *launches = nl;
    return FPM_OK;
  }
  if (mode == FPM_RUN_PLAIN) {
    // one tile at a time, one LED per launch
    for (int t = 0; t < p->n_tiles; ++t) {
      for (int s = 0; s < sl.n_steps; ++s) {
        const long long i0 = sl.step_off[s], i1 = sl.step_off[s + 1];
        // items of step s are sorted by tile
        const int32_t *it = sl.items.data();
        long long lo = i0, hi = i1;
        while (lo < hi && it[lo * 4] < t) ++lo;
        long long e = lo;
        while (e < hi && it[e * 4] == t) ++e;
        if (e == lo) continue;
        for (long long k = lo; k < e; ++k) {
          if ((rc = launch_update(p, a, k, 1, st))) return rc;
          ++nl;
        }
        if (p->epry) {
          for (long long k = sl.merge_off[s]; k < sl.merge_off[s + 1]; ++k)
            if (sl.merges[k * 2] == t) {
              if ((rc = launch_merge(d->pup, d->dpup, sd->merges + k, 1, p->y_lo, rows, p->m,
                                     p->max_width, p->disc_ok ? 1 : 0, st)))
                return rc;
              ++nl;
            }
        }
      }
    }
    FPM_CK(cudaGetLastError());
    *launches = nl;
    return FPM_OK;
  }
  return fail(FPM_EINVAL, "unknown mode %d", mode);
}

// FPM_ETIMEOUT if the last persistent run's bounded wait gave up (synchronises).
static int device_error(fpm_plan *p) {
  DeviceState *d = p->dev;
  if (!d || !d->err) return FPM_OK;
  unsigned e[2] = {0, 0};
  FPM_CK(cudaDeviceSynchronize());
  FPM_CK(cudaMemcpy(e, d->err, sizeof(e), cudaMemcpyDeviceToHost));
  if (e[0]) return fail(FPM_ETIMEOUT, "a bounded device wait of the persistent kernel gave up (error bits 0x%x)", e[0]);
  return FPM_OK;
}

int run_persistent(fpm_plan *p, int32_t iters, cudaStream_t st, bool graph, bool stall_test) {
  DeviceState *d = p->dev;
  auto it = d->queues.find(iters);
  if (it == d->queues.end()) {
    QueueDev *q = nullptr;
    int rc = make_queue({QueueJob{p, iters}}, &q);
    if (rc) return rc;
    it = d->queues.emplace(iters, q).first;
  }
  QueueDev *q = it->second;
  if (!graph || stall_test) {
    int rc = launch_queue(q, d->err, stall_test ? 1 : 0, st, &d->persistent_clusters);
    d->run_launches = 1;
    return rc;
  }
  GraphKey key{iters, FPM_RUN_PERSISTENT | FPM_RUN_GRAPH, st};
  auto g = d->graphs.find(key);
  if (g == d->graphs.end()) {
    cudaStream_t cap = st;
    bool own = false;
    if (cap == nullptr) {
      FPM_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      own = true;
    }
    FPM_CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    int rc = launch_queue(q, d->err, 0, cap, &d->persistent_clusters);
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &gr);
    if (own) cudaStreamDestroy(cap);
    if (rc) {
      if (gr) cudaGraphDestroy(gr);
      return rc;
    }
    if (e != cudaSuccess) return fail(FPM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return fail(FPM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    g = d->graphs.emplace(key, ex).first;
  }
  FPM_CK(cudaGraphLaunch(g->second, st));
  d->run_launches = 1;
  return FPM_OK;
}

// Batches of several plans: one queue per distinct batch (cached by its plans and
// loop counts), the error words of every plan reset and pointed at the first's.
struct BatchKey {
  std::vector<fpm_plan *> plans;
  std::vector<int32_t> iters;
  cudaStream_t st;
  bool graph;
  int mode = FPM_RUN_PERSISTENT;
  bool operator<(const BatchKey &o) const {
    if (plans != o.plans) return plans < o.plans;
    if (iters != o.iters) return iters < o.iters;
    if (st != o.st) return st < o.st;
    if (mode != o.mode) return mode < o.mode;
    return graph < o.graph;
  }
};
struct BatchEntry {
  QueueDev *q = nullptr;
  cudaGraphExec_t exec = nullptr;
};
static std::mutex g_batch_mu;
static std::map<BatchKey, BatchEntry> g_batches;

void forget_batches(fpm_plan *p) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (auto it = g_batches.begin(); it != g_batches.end();) {
    if (std::find(it->first.plans.begin(), it->first.plans.end(), p) != it->first.plans.end()) {
      if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
      if (it->second.q) free_queue(it->second.q);
      it = g_batches.erase(it);
    } else {
      ++it;
    }
  }
}

// Every plan's wave steps on its own stream (each possibly forked into its tile
// branches), forked from and joined back into st.
static int enqueue_batch_waves(const std::vector<QueueJob> &jobs, cudaStream_t st, int64_t *launches) {
  DeviceState *d0 = jobs[0].plan->dev;
  for (const QueueJob &j : jobs) {
    DeviceState *d = j.plan->dev;
    if (!d->batch_st) FPM_CK(cudaStreamCreateWithFlags(&d->batch_st, cudaStreamNonBlocking));
    for (cudaEvent_t &ev : d->batch_ev)
      if (!ev) FPM_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  FPM_CK(cudaEventRecord(d0->batch_ev[0], st));             // fork
  int rc = FPM_OK;
  for (const QueueJob &j : jobs) {
    DeviceState *d = j.plan->dev;
    FPM_CK(cudaStreamWaitEvent(d->batch_st, d0->batch_ev[0], 0));
    if (rc == FPM_OK) {
      const int b = std::min(d->branches, std::max(1, j.plan->n_tiles));
      rc = b > 1 ? enqueue_wave_branches(j.plan, j.iters, 0, 1 << 30, b, d->batch_st, launches)
                 : enqueue_wave_tiles(j.plan, j.iters, 0, 1 << 30, 0, j.plan->n_tiles, d->batch_st, launches);
    }
    FPM_CK(cudaEventRecord(d->batch_ev[1], d->batch_st));   // join
    FPM_CK(cudaStreamWaitEvent(st, d->batch_ev[1], 0));
  }
  return rc;
}

// A batch of plans run wave by wave, each plan an independent part of one graph
// (cached per batch) or, without a graph, of the stream's work.
int run_batch_waves(const std::vector<QueueJob> &jobs, cudaStream_t st, bool graph) {
  int64_t nl = 0;
  if (!graph) return enqueue_batch_waves(jobs, st, &nl);
  BatchKey key;
  for (const QueueJob &j : jobs) {
    key.plans.push_back(j.plan);
    key.iters.push_back(j.iters);
  }
  key.st = st;
  key.graph = true;
  key.mode = FPM_RUN_WAVES;
  std::lock_guard<std::mutex> lk(g_batch_mu);
  auto it = g_batches.find(key);
  if (it == g_batches.end()) {
    for (const QueueJob &j : jobs) {                            // step lists outside the capture
      const StepLists &sl = step_lists(j.plan, j.iters);
      int rc = 0;
      if (!device_steps(j.plan, j.iters, sl, &rc)) return rc;
    }
    cudaStream_t cap = st;
    bool own = false;
    if (cap == nullptr) {
      FPM_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      own = true;
    }
    FPM_CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_batch_waves(jobs, cap, &nl);
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &gr);
    if (own) cudaStreamDestroy(cap);
    if (rc) {
      if (gr) cudaGraphDestroy(gr);
      return rc;
    }
    if (e != cudaSuccess) return fail(FPM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    BatchEntry be;
    e = cudaGraphInstantiate(&be.exec, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return fail(FPM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    it = g_batches.emplace(key, be).first;
  }
  FPM_CK(cudaGraphLaunch(it->second.exec, st));
  return FPM_OK;
}

int run_batch(const std::vector<QueueJob> &jobs, cudaStream_t st, bool graph) {
  BatchKey key;
  for (const QueueJob &j : jobs) {
    key.plans.push_back(j.plan);
    key.iters.push_back(j.iters);
  }
  key.st = st;
  key.graph = graph;
  std::lock_guard<std::mutex> lk(g_batch_mu);
  auto it = g_batches.find(key);
  if (it == g_batches.end()) {
    BatchEntry e;
    int rc = make_queue(jobs, &e.q);
    if (rc) return rc;
    it = g_batches.emplace(key, e).first;
  }
  BatchEntry &e = it->second;
  unsigned *err = jobs[0].plan->dev->err;
  for (size_t k = 1; k < jobs.size(); ++k)
    FPM_CK(cudaMemsetAsync(jobs[k].plan->dev->err, 0, 4 * sizeof(unsigned), st));
  int clusters = 0;
  if (!graph) {
    int rc = launch_queue(e.q, err, 0, st, &clusters);
    if (rc) return rc;
  } else {
    if (!e.exec) {
      cudaStream_t cap = st;
      bool own = false;
      if (cap == nullptr) {
        FPM_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        own = true;
      }
      FPM_CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
      int rc = launch_queue(e.q, err, 0, cap, &clusters);
      cudaGraph_t gr = nullptr;
      cudaError_t ce = cudaStreamEndCapture(cap, &gr);
      if (own) cudaStreamDestroy(cap);
      if (rc) {
        if (gr) cudaGraphDestroy(gr);
        return rc;
      }
      if (ce != cudaSuccess) return fail(FPM_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
      ce = cudaGraphInstantiate(&e.exec, gr, 0);
      cudaGraphDestroy(gr);
      if (ce != cudaSuccess) return fail(FPM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
    }
    FPM_CK(cudaGraphLaunch(e.exec, st));
  }
  // the batch reports its device errors through the first plan; copy the word to the others
  for (size_t k = 1; k < jobs.size(); ++k)
    FPM_CK(cudaMemcpyAsync(jobs[k].plan->dev->err, err, 2 * sizeof(unsigned), cudaMemcpyDeviceToDevice, st));
  for (const QueueJob &j : jobs) {
    j.plan->dev->run_launches = 1;
    if (clusters) j.plan->dev->persistent_clusters = clusters;
  }
  return FPM_OK;
}

int get_stats(fpm_plan *p, fpm_stats *out) {
  std::memset(out, 0, sizeof(*out));
  DeviceState *d = p->dev;
  if (!d) return FPM_OK;
  out->load_launches = d->load_launches;
  out->run_launches = d->run_launches;
  out->persistent_clusters = d->persistent_clusters;
  out->run_threads = d->run_threads;
  out->run_cluster = d->run_cluster;
  out->run_lanes = d->run_lanes;
  out->pad0 = 0;
  online_progress(p, &out->online_launched, &out->online_steps);
  const int derr = device_error(p);
  out->device_error = derr == FPM_ETIMEOUT ? FPM_ETIMEOUT : 0;
  if (d->timed_valid && !d->timed_steps.empty()) {
    const size_t last = d->events.size() > 0 ? (size_t)(2 * d->timed_n_steps) : 0;
    FPM_CK(cudaEventSynchronize(d->events[last]));
    double ms = 0, mms = 0;
    for (size_t k = 0; k < d->timed_steps.size(); ++k) {
      const int64_t s = d->timed_steps[k];
      float f = 0.f, g = 0.f;
      FPM_CK(cudaEventElapsedTime(&f, d->events[2 * s], d->events[2 * s + 1]));
      const cudaEvent_t next = k + 1 < d->timed_steps.size() ? d->events[2 * d->timed_steps[k + 1]] : d->events[last];
      FPM_CK(cudaEventElapsedTime(&g, d->events[2 * s + 1], next));
      ms += f;
      mms += g;
    }
    out->update_ms = ms;
    out->merge_ms = mms;
    out->update_launches = (int64_t)d->timed_steps.size();
    out->updates = d->timed_updates;
  }
  return derr;
}

}  // namespace fpm

using fpm::fail;

extern "C" {

int fpm_load_tiles(fpm_plan *p, const void *stack, int32_t dtype, int32_t on_device, int64_t stride_led,
                   int64_t stride_row, float counts_per_unit, void *stream) {
  fpm::clear_error();
  if (!p || !stack) return fail(FPM_EINVAL, "fpm_load_tiles: null argument");
  if (p->busy) return fail(FPM_EBUSY, "plan is owned by a server job");
  return fpm::load_tiles(p, stack, dtype, on_device, stride_led, stride_row, counts_per_unit, (cudaStream_t)stream);
}

}  // extern "C"

namespace fpm {

int validate_stack(fpm_plan *p, const void *stack, int32_t dtype, int64_t stride_led, int64_t stride_row,
                   float counts_per_unit, size_t *bytes) {
  if (dtype != FPM_U16 && dtype != FPM_F32) return fail(FPM_EINVAL, "unknown image dtype %d", dtype);
  if (!(counts_per_unit > 0) || !std::isfinite(counts_per_unit))
    return fail(FPM_EINVAL, "counts_per_unit must be positive and finite");
  const int64_t es = dtype == FPM_U16 ? 2 : 4;
  if (stride_row < p->sensor_w || stride_led < stride_row * p->sensor_h)
    return fail(FPM_EINVAL, "strides (%lld, %lld) smaller than the image", (long long)stride_led, (long long)stride_row);
  if ((stride_row * es) % 16 || (stride_led * es) % 16 || ((uintptr_t)stack % 16))
    return fail(FPM_EINVAL, "stack base, rows and LED planes must be 16-byte aligned");
  if (bytes)
    *bytes = (size_t)((p->n_leds - 1) * stride_led + (int64_t)(p->sensor_h - 1) * stride_row + p->sensor_w) * es;
  return FPM_OK;
}

// The tile-image buffer for images of type dtype (reallocated, with the launch
// caches that hold its address, when the size changes).
int ensure_images(fpm_plan *p, int32_t dtype) {
  DeviceState *d = p->dev;
  const size_t ib = image_bytes(p, dtype);
  if (d->images_bytes != ib) {
    // queues and graphs hold the image address: drop them with the old buffer
    cudaDeviceSynchronize();
    for (auto &kv : d->graphs) cudaGraphExecDestroy(kv.second);
    d->graphs.clear();
    d->graph_launches.clear();
    for (auto &kv : d->queues) free_queue(kv.second);
    d->queues.clear();
    forget_batches(p);
    if (d->images) cudaFree(d->images);
    d->images = nullptr;
    d->images_bytes = 0;
    d->loaded = false;
    if (cudaMalloc(&d->images, ib) != cudaSuccess) {
      cudaGetLastError();
      return fail(FPM_ENOMEM, "device allocation of the tile images (%zu bytes) failed", ib);
    }
    d->images_bytes = ib;
  }
  return FPM_OK;
}

// Gather n_src sensor images (LEDs led0 ..) into the tile-image buffer.
int gather_tile_images(fpm_plan *p, const void *src, int32_t dtype, long long stride_led, long long stride_row,
                       int led0, int n_src, cudaStream_t st) {
  DeviceState *d = p->dev;
  const cudaError_t e =
      dtype == FPM_U16
          ? launch_tile_images((uint16_t *)d->images, (const uint16_t *)src, stride_led, stride_row, d->origins, p->m,
                               p->n_tiles, p->n_leds, led0, n_src, st)
          : launch_tile_images((float *)d->images, (const float *)src, stride_led, stride_row, d->origins, p->m,
                               p->n_tiles, p->n_leds, led0, n_src, st);
  if (e != cudaSuccess) return fail(FPM_ECUDA, "tile image gather: %s", cudaGetErrorString(e));
  return FPM_OK;
}

int begin_load(fpm_plan *p, int32_t dtype, float counts_per_unit, cudaStream_t st) {
  DeviceState *d = p->dev;
  d->loaded = false;
  d->dtype = dtype;
  d->inv_counts = 1.0f / counts_per_unit;
  FPM_CK(cudaMemsetAsync(d->err, 0, 4 * sizeof(unsigned), st));   // a reload clears a previous failure
  return FPM_OK;
}

void mark_loaded(fpm_plan *p) { p->dev->loaded = true; }

int load_tiles(fpm_plan *p, const void *stack, int32_t dtype, int32_t on_device, int64_t stride_led,
               int64_t stride_row, float counts_per_unit, cudaStream_t st) {
  if (!stack) return fail(FPM_EINVAL, "fpm_load_tiles: null stack");
  size_t bytes = 0;
  int rc = validate_stack(p, stack, dtype, stride_led, stride_row, counts_per_unit, &bytes);
  if (rc) return rc;
  if ((rc = ensure_device_state(p))) return rc;
  DeviceState *d = p->dev;
  if ((rc = ensure_images(p, dtype))) return rc;
  const void *src = stack;
  void *staging = nullptr;        // a host stack passes through device memory once, for the gather
  if (on_device) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, stack) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      return fail(FPM_EINVAL, "on_device stack is not device memory");
    }
  } else {
    if (cudaMallocAsync(&staging, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      return fail(FPM_ENOMEM, "device staging of the image stack (%zu bytes) failed", bytes);
    }
    FPM_CK(cudaMemcpyAsync(staging, stack, bytes, cudaMemcpyHostToDevice, st));
    src = staging;
  }
  if ((rc = begin_load(p, dtype, counts_per_unit, st))) return rc;
  // every tile's images in the update kernel's column layout, then the initial guess
  rc = gather_tile_images(p, src, dtype, stride_led, stride_row, 0, p->n_leds, st);
  if (!rc) {
    const size_t es = dtype == FPM_U16 ? 2 : 4;
    rc = run_init(p, static_cast<const char *>(src) + (size_t)p->order[0] * stride_led * es, stride_row, st);
  }
  if (staging) cudaFreeAsync(staging, st);
  if (rc) return rc;
  d->loaded = true;
  return FPM_OK;
}

size_t image_bytes(const fpm_plan *p, int32_t dtype) {
  return (size_t)p->n_tiles * p->n_leds * p->m * p->m * (dtype == FPM_U16 ? 2 : 4);
}

size_t plan_device_bytes(const fpm_plan *p, int32_t dtype) {
  const size_t T = p->n_tiles, n = p->n, m = p->m;
  return T * n * n * 8 + T * m * m * 8 * (p->epry ? 2 + (size_t)p->max_width : 2) + image_bytes(p, dtype);
}

}  // namespace fpm

extern "C" {

int fpm_reconstruct(fpm_plan *p, int32_t iters, int32_t mode, void *stream) {
  fpm::clear_error();
  if (!p) return fail(FPM_EINVAL, "fpm_reconstruct: null plan");
  if (p->busy) return fail(FPM_EBUSY, "plan is owned by a server job");
  if (!p->dev || !p->dev->loaded) return fail(FPM_ESTATE, "fpm_reconstruct before fpm_load_tiles");
  if (iters < 1 || iters > p->iters) return fail(FPM_EINVAL, "iters %d outside 1..%d", iters, p->iters);
  int base = mode & 0xff;
  const bool graph = (mode & FPM_RUN_GRAPH) != 0;
  const bool timed = (mode & FPM_RUN_TIMED) != 0;
  const bool stall = (mode & FPM_RUN_FAULT_TEST) != 0;
  if ((mode & ~(0xff | FPM_RUN_GRAPH | FPM_RUN_TIMED | FPM_RUN_FAULT_TEST)) ||
      (base != FPM_RUN_PLAIN && base != FPM_RUN_WAVES && base != FPM_RUN_PERSISTENT && base != FPM_RUN_AUTO))
    return fail(FPM_EINVAL, "unknown mode 0x%x", mode);
  if (base == FPM_RUN_AUTO) {
    base = p->dev->tuned_mode;
    mode = (mode & ~0xff) | base;
  }
  if (timed && base != FPM_RUN_WAVES) return fail(FPM_EINVAL, "FPM_RUN_TIMED needs FPM_RUN_WAVES");
  if (stall && base != FPM_RUN_PERSISTENT) return fail(FPM_EINVAL, "FPM_RUN_FAULT_TEST needs FPM_RUN_PERSISTENT");
  cudaStream_t st = (cudaStream_t)stream;
  fpm::DeviceState *d = p->dev;
  if (base == FPM_RUN_PERSISTENT) {
    d->run_threads = fpm::persistent_block_threads(p->m);
    d->run_cluster = fpm::persistent_cluster_size(p->m);
    d->run_lanes = fpm::persistent_lanes(p->m);
    return fpm::run_persistent(p, iters, st, graph, stall);
  }
  if (!graph) {
    int64_t nl = 0;
    int rc = fpm::enqueue_reconstruct(p, iters, base, st, timed, false, &nl);
    d->run_launches = nl;
    d->run_threads = d->var->t;
    d->run_cluster = d->var->c;
    d->run_lanes = d->var->tpt;
    return rc;
  }
  const int branches = (base == FPM_RUN_WAVES && !timed) ? std::min(d->branches, std::max(1, p->n_tiles)) : 1;
  fpm::GraphKey key{iters, (mode & 0xfff) | (branches << 12), st};
  auto it = d->graphs.find(key);
  if (it == d->graphs.end()) {
    // build step lists and device copies outside the capture
    const fpm::StepLists &sl = fpm::step_lists(p, iters);
    int rc = 0;
    if (!fpm::device_steps(p, iters, sl, &rc)) return rc;
    cudaStream_t cap = st;
    bool own = false;
    if (cap == nullptr) {
      FPM_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      own = true;
    }
    FPM_CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    int64_t nl = 0;
    if (branches > 1) rc = fpm::enqueue_wave_branches(p, iters, 0, 1 << 30, branches, cap, &nl);
    else rc = fpm::enqueue_reconstruct(p, iters, base, cap, timed, true, &nl);
    d->graph_launches[key] = nl;
    d->graph_threads[key] = d->var->t;
    d->graph_cluster[key] = d->var->c;
    d->graph_lanes[key] = d->var->tpt;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (own) cudaStreamDestroy(cap);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return fail(FPM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(FPM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    it = d->graphs.emplace(key, ex).first;
  }
  if (timed) {
    // the events of this graph belong to its capture-time schedule
    const fpm::StepLists &sl = fpm::step_lists(p, iters);
    d->timed_steps.clear();
    d->timed_updates = 0;
    d->timed_n_steps = sl.n_steps;
    for (int s = 0; s < sl.n_steps; ++s)
      if (sl.step_off[s + 1] > sl.step_off[s]) {
        d->timed_steps.push_back(s);
        d->timed_updates += sl.step_off[s + 1] - sl.step_off[s];
      }
    d->timed_valid = true;
  }
  FPM_CK(cudaGraphLaunch(it->second, st));
  d->run_launches = d->graph_launches[key];
  d->run_threads = d->graph_threads[key];
  d->run_cluster = d->graph_cluster[key];
  d->run_lanes = d->graph_lanes[key];
  return FPM_OK;
}

int fpm_reconstruct_batch(fpm_plan *const *plans, const int32_t *iters, int32_t n, int32_t mode, void *stream) {
  fpm::clear_error();
  if (!plans || !iters || n < 1) return fail(FPM_EINVAL, "fpm_reconstruct_batch: empty batch");
  const int base = mode & ~FPM_RUN_GRAPH;
  if (base != FPM_RUN_PERSISTENT && base != FPM_RUN_WAVES)
    return fail(FPM_EINVAL, "fpm_reconstruct_batch runs FPM_RUN_PERSISTENT or FPM_RUN_WAVES (optionally | FPM_RUN_GRAPH)");
  std::vector<fpm::QueueJob> jobs;
  for (int i = 0; i < n; ++i) {
    fpm_plan *p = plans[i];
    if (!p) return fail(FPM_EINVAL, "plan %d is null", i);
    if (p->busy) return fail(FPM_EBUSY, "plan %d is owned by a server job", i);
    if (!p->dev || !p->dev->loaded) return fail(FPM_ESTATE, "plan %d is not loaded", i);
    if (iters[i] < 1 || iters[i] > p->iters) return fail(FPM_EINVAL, "plan %d: iters %d outside 1..%d", i, iters[i], p->iters);
    for (int k = 0; k < i; ++k)
      if (plans[k] == p) return fail(FPM_EINVAL, "plan %d appears twice", i);
    jobs.push_back(fpm::QueueJob{p, iters[i]});
  }
  if (base == FPM_RUN_WAVES) return fpm::run_batch_waves(jobs, (cudaStream_t)stream, (mode & FPM_RUN_GRAPH) != 0);
  return fpm::run_batch(jobs, (cudaStream_t)stream, (mode & FPM_RUN_GRAPH) != 0);
}

int fpm_autotune(fpm_plan *p, int32_t iters, void *stream, fpm_tune_entry *entries, int32_t max_entries,
                 int32_t *n_entries, int32_t *best) {
  fpm::clear_error();
  if (!p) return fail(FPM_EINVAL, "fpm_autotune: null plan");
  if (p->busy) return fail(FPM_EBUSY, "plan is owned by a server job");
  if (!p->dev || !p->dev->loaded) return fail(FPM_ESTATE, "fpm_autotune before fpm_load_tiles");
  if (iters < 1 || iters > p->iters) return fail(FPM_EINVAL, "iters %d outside 1..%d", iters, p->iters);
  fpm::DeviceState *d = p->dev;
  cudaStream_t st = (cudaStream_t)stream;
  const int rows = p->y_hi - p->y_lo + 1;
  const size_t sb = (size_t)p->n_tiles * p->n * p->n * sizeof(float2);
  const size_t pb = (size_t)p->n_tiles * p->m * p->m * sizeof(float2);
  void *save = nullptr;
  FPM_CK(cudaMalloc(&save, sb + pb));
  struct Cand {
    int mode;
    const fpm::Variant *v;
    int branches;
    double ms;
  };
  std::vector<Cand> cands;
  for (const auto &v : fpm::variants())
    if (v.m == p->m && v.smem(rows) <= fpm::kMaxSmem) {
      cands.push_back({FPM_RUN_WAVES, &v, 1, 0.0});
      for (int b : {2, 4, 8})
        if (b <= p->n_tiles) cands.push_back({FPM_RUN_WAVES, &v, b, 0.0});
    }
  if (fpm::persistent_fits(p->m, rows)) cands.push_back({FPM_RUN_PERSISTENT, nullptr, 1, 0.0});
  const fpm::Variant *keep = d->var;
  const int32_t keep_branches = d->branches;
  int rc = FPM_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = fail(FPM_ECUDA, "events");
  if (rc == FPM_OK && (cudaMemcpyAsync(save, d->spec, sb, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                       cudaMemcpyAsync((char *)save + sb, d->pup, pb, cudaMemcpyDeviceToDevice, st) != cudaSuccess))
    rc = fail(FPM_ECUDA, "saving the state");
  for (auto &c : cands) {
    if (rc) break;
    if (c.v) {
      d->var = c.v;
      d->branches = c.branches;
      for (auto &kv : d->graphs) cudaGraphExecDestroy(kv.second);   // graphs hold the previous variant
      d->graphs.clear();
    }
    for (int rep_ = 0; rep_ < 2 && rc == FPM_OK; ++rep_) {          // warm-up (graph capture), then timed
      if (rep_ == 1 && cudaEventRecord(e0, st) != cudaSuccess) rc = fail(FPM_ECUDA, "event");
      if (rc == FPM_OK) rc = fpm_reconstruct(p, iters, c.mode | FPM_RUN_GRAPH, stream);
      if (rc == FPM_OK && rep_ == 1 && cudaEventRecord(e1, st) != cudaSuccess) rc = fail(FPM_ECUDA, "event");
      if (rc == FPM_OK && (cudaMemcpyAsync(d->spec, save, sb, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                           cudaMemcpyAsync(d->pup, (char *)save + sb, pb, cudaMemcpyDeviceToDevice, st) != cudaSuccess))
        rc = fail(FPM_ECUDA, "restoring the state");
    }
    float ms = 0.f;
    if (rc == FPM_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = fail(FPM_ECUDA, "timing");
    c.ms = ms;
    if (!c.v) d->var = keep;
  }
  int bi = 0;
  for (size_t i = 0; i < cands.size(); ++i)
    if (cands[i].ms < cands[bi].ms) bi = (int)i;
  if (rc == FPM_OK) {
    // the fastest wave variant serves FPM_RUN_WAVES; the fastest path serves FPM_RUN_AUTO
    int bw = -1;
    for (size_t i = 0; i < cands.size(); ++i)
      if (cands[i].v && (bw < 0 || cands[i].ms < cands[bw].ms)) bw = (int)i;
    if (bw >= 0) {
      d->var = cands[bw].v;
      d->branches = cands[bw].branches;
    } else {
      d->branches = keep_branches;
    }
    d->tuned_mode = cands[bi].mode;
    p->cluster = d->var->c;
    p->threads = d->var->t;
  } else {
    d->var = keep;
    d->branches = keep_branches;
  }
  // the candidates' wave graphs share one cache key: whichever ran last must not
  // outlive the tuning, so the chosen variant's graph is captured on next use
  cudaStreamSynchronize(st);
  for (auto &kv : d->graphs) cudaGraphExecDestroy(kv.second);
  d->graphs.clear();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(save);
  if (rc) return rc;
  if (n_entries) *n_entries = (int32_t)std::min<size_t>(cands.size(), (size_t)std::max(0, max_entries));
  if (entries)
    for (int i = 0; i < (int)cands.size() && i < max_entries; ++i) {
      const auto &c = cands[i];
      entries[i].mode = c.mode;
      entries[i].threads = c.v ? c.v->t : fpm::persistent_block_threads(p->m);
      entries[i].cluster = c.v ? c.v->c : fpm::persistent_cluster_size(p->m);
      entries[i].branches = c.branches;
      entries[i].ms = c.ms;
      int va = 0, vb = 0, vc = 0, vt = 0;
      fpm::update_variant(p->m, rows, &va, &vb, &vc, &vt);          // the persistent kernel's split is the same
      entries[i].lanes = c.v ? c.v->tpt : fpm::persistent_lanes(p->m);
      entries[i].radix_a = c.v ? c.v->a : va;
      entries[i].radix_b = c.v ? c.v->b : vb;
      entries[i].pad0 = 0;
    }
  if (best) *best = bi;
  return FPM_OK;
}

int fpm_get_stats(fpm_plan *p, fpm_stats *out) {
  if (!p || !out) return fail(FPM_EINVAL, "fpm_get_stats: null argument");
  return fpm::get_stats(p, out);
}

static int copy_out(fpm_plan *p, const void *src, void *dst, size_t bytes, int32_t on_device, cudaStream_t st) {
  FPM_CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  if (!on_device) {
    FPM_CK(cudaStreamSynchronize(st));
    unsigned e = 0;
    FPM_CK(cudaMemcpy(&e, p->dev->err, sizeof(e), cudaMemcpyDeviceToHost));
    if (e) return fail(FPM_ETIMEOUT, "a bounded device wait of the last persistent run gave up");
  }
  return FPM_OK;
}

int fpm_get_spectrum(fpm_plan *p, int32_t tile, void *dst, int32_t on_device, void *stream) {
  fpm::clear_error();
  if (!p || !dst) return fail(FPM_EINVAL, "fpm_get_spectrum: null argument");
  if (tile < 0 || tile >= p->n_tiles) return fail(FPM_EINVAL, "tile %d out of range", tile);
  if (!p->dev || !p->dev->loaded) return fail(FPM_ESTATE, "no state before fpm_load_tiles");
  const size_t nn = (size_t)p->n * p->n;
  return copy_out(p, p->dev->spec + (size_t)tile * nn, dst, nn * sizeof(float2), on_device, (cudaStream_t)stream);
}

int fpm_get_spectra(fpm_plan *p, void *dst, int32_t on_device, void *stream) {
  fpm::clear_error();
  if (!p || !dst) return fail(FPM_EINVAL, "fpm_get_spectra: null argument");
  if (!p->dev || !p->dev->loaded) return fail(FPM_ESTATE, "no state before fpm_load_tiles");
  const size_t bytes = (size_t)p->n_tiles * p->n * p->n * sizeof(float2);
  FPM_CK(cudaMemcpyAsync(dst, p->dev->spec, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                         (cudaStream_t)stream));
  return FPM_OK;
}

int fpm_get_pupil(fpm_plan *p, int32_t tile, void *dst, int32_t on_device, void *stream) {
  fpm::clear_error();
  if (!p || !dst) return fail(FPM_EINVAL, "fpm_get_pupil: null argument");
  if (tile < 0 || tile >= p->n_tiles) return fail(FPM_EINVAL, "tile %d out of range", tile);
  if (!p->dev || !p->dev->loaded) return fail(FPM_ESTATE, "no state before fpm_load_tiles");
  const size_t mm = (size_t)p->m * p->m;
  return copy_out(p, p->dev->pup + (size_t)tile * mm, dst, mm * sizeof(float2), on_device, (cudaStream_t)stream);
}

int fpm_set_state(fpm_plan *p, int32_t tile, const void *spectrum, const void *pupil, void *stream) {
  fpm::clear_error();
  if (!p) return fail(FPM_EINVAL, "fpm_set_state: null plan");
  if (tile < 0 || tile >= p->n_tiles) return fail(FPM_EINVAL, "tile %d out of range", tile);
  if (!p->dev || !p->dev->loaded) return fail(FPM_ESTATE, "fpm_set_state before fpm_load_tiles");
  cudaStream_t st = (cudaStream_t)stream;
  fpm::DeviceState *d = p->dev;
  const size_t nn = (size_t)p->n * p->n, mm = (size_t)p->m * p->m;
  if (spectrum) FPM_CK(cudaMemcpyAsync(d->spec + tile * nn, spectrum, nn * 8, cudaMemcpyHostToDevice, st));
  if (pupil) FPM_CK(cudaMemcpyAsync(d->pup + tile * mm, pupil, mm * 8, cudaMemcpyHostToDevice, st));
  FPM_CK(cudaStreamSynchronize(st));
  return FPM_OK;
}

int fpm_simulate(fpm_plan *p, const void *objects, float *out, void *stream) {
  fpm::clear_error();
  if (!p || !objects || !out) return fail(FPM_EINVAL, "fpm_simulate: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int m = p->m, n = p->n, T = p->n_tiles, L = p->n_leds;
  std::vector<int2> sh((size_t)T * L);
  for (size_t i = 0; i < sh.size(); ++i) sh[i] = make_int2(p->shifts[i * 2], p->shifts[i * 2 + 1]);
  float2 *spec = nullptr, *box = nullptr, *pup = nullptr, *twn = nullptr, *twm = nullptr;
  int2 *dsh = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    for (void *q : {(void *)spec, (void *)box, (void *)pup, (void *)twn, (void *)twm, (void *)dsh}) fpm::dfree(q);
  };
  int rc = FPM_OK;
  do {
    cudaError_t e;
    if ((e = cudaMalloc((void **)&spec, (size_t)T * n * n * 8)) != cudaSuccess ||
        (e = cudaMalloc((void **)&box, (size_t)T * m * m * 8)) != cudaSuccess ||
        (e = cudaMalloc((void **)&pup, (size_t)T * m * m * 8)) != cudaSuccess ||
        (e = cudaMalloc((void **)&dsh, sh.size() * sizeof(int2))) != cudaSuccess ||
        (e = cudaMalloc((void **)&twn, (size_t)n * 8)) != cudaSuccess ||
        (e = cudaMalloc((void **)&twm, (size_t)m * 8)) != cudaSuccess) {
      rc = fail(FPM_ENOMEM, "fpm_simulate: device allocation failed: %s", cudaGetErrorString(e));
      break;
    }
    std::vector<float2> tn = fpm::twiddles_line(n, -1), tm = fpm::twiddles_line(m, +1);
    if (cudaMemcpy(twn, tn.data(), tn.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(twm, tm.data(), tm.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dsh, sh.data(), sh.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(pup, p->pupil0.data(), (size_t)T * m * m * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = fail(FPM_ECUDA, "fpm_simulate: upload failed");
      break;
    }
    if (cudaMemcpyAsync(spec, objects, (size_t)T * n * n * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      rc = fail(FPM_ECUDA, "fpm_simulate: objects must be device memory");
      break;
    }
    if ((rc = fpm::launch_fft_lines(spec, twn, n, -1, (long long)T * n, n, (long long)n * n, n, 1, st))) break;
    if ((rc = fpm::launch_fft_lines(spec, twn, n, -1, (long long)T * n, n, (long long)n * n, 1, n, st))) break;
    const long long tot = (long long)T * m * m;
    const float inv_n2 = (float)(1.0 / ((double)n * n));
    for (int l = 0; l < L && rc == FPM_OK; ++l) {
      fpm::sim_crop_kernel<<<fpm::grid_for(tot, 256), 256, 0, st>>>(box, spec, pup, dsh, l, L, m, n, T);
      if ((rc = fpm::launch_fft_lines(box, twm, m, +1, (long long)T * m, m, (long long)m * m, m, 1, st))) break;
      if ((rc = fpm::launch_fft_lines(box, twm, m, +1, (long long)T * m, m, (long long)m * m, 1, m, st))) break;
      fpm::sim_abs_kernel<<<fpm::grid_for(tot, 256), 256, 0, st>>>(out, box, l, L, m, T, inv_n2);
    }
    if (rc == FPM_OK && cudaGetLastError() != cudaSuccess) rc = fail(FPM_ECUDA, "fpm_simulate: launch failed");
  } while (0);
  cleanup();
  return rc;
}

}  // extern "C"
