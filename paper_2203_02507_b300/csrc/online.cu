// Online reconstruction: LR images ingested one at a time while they are being
// acquired (Sec. 3.4, Fig. 7(a)), each one's tile updates started at once.
//
// The schedule is the plan's wave schedule for `iters` loops, unchanged: a wave
// step may run once every LED it updates has arrived, and steps run in their
// order.  Each step needs a prefix of the LED order (its largest order position
// plus one, made non-decreasing along the steps); a push extends the arrived
// prefix and launches every step that became ready.  Pushes may come in any
// order; with images in the order of the LED sequence (the acquisition order)
// the first loop's waves run as the images come in, and fpm_online_finish runs
// the rest.  The result is bit-identical to fpm_load_tiles + fpm_reconstruct
// (FPM_RUN_WAVES) on the same images.
//
// A host image is copied on the plan's own copy stream into one of four staging
// buffers (events order it before the gather that reads it and the next copy
// into the same buffer after that gather), so with page-locked host memory the
// copy overlaps the updates running on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "runtime.h"

namespace fpm {

#define FPM_CK(call)                                                                         \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(FPM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

constexpr int kOnlineRing = 4;

struct OnlineState {
  int32_t iters = 0, dtype = FPM_U16;
  bool active = false;
  std::vector<int32_t> pos;          // order position of each LED index
  std::vector<uint8_t> arrived;      // per LED index
  int32_t prefix = 0;                // order positions [0, prefix) have all arrived
  std::vector<int32_t> need;         // per wave step: arrived prefix it needs (non-decreasing)
  int32_t launched = 0;              // wave steps enqueued
  int64_t pushes = 0;
  void *staging[kOnlineRing] = {};
  size_t staging_bytes = 0;
  cudaEvent_t copied[kOnlineRing] = {}, freed[kOnlineRing] = {};
  bool used[kOnlineRing] = {};
  cudaStream_t copy = nullptr;
  // the steps the last image of an in-order ingestion releases, captured as a
  // graph with tile branches at fpm_online_begin
  cudaGraphExec_t tail = nullptr;
  int32_t tail_from = -1;
};

void destroy_online_state(fpm_plan *p) {
  OnlineState *o = p->online;
  if (!o) return;
  if (o->copy) cudaStreamSynchronize(o->copy);
  for (int k = 0; k < kOnlineRing; ++k) {
    if (o->freed[k]) cudaEventSynchronize(o->freed[k]);
    if (o->staging[k]) cudaFree(o->staging[k]);
    if (o->copied[k]) cudaEventDestroy(o->copied[k]);
    if (o->freed[k]) cudaEventDestroy(o->freed[k]);
  }
  if (o->copy) cudaStreamDestroy(o->copy);
  if (o->tail) cudaGraphExecDestroy(o->tail);
  delete o;
  p->online = nullptr;
}

static int online_resources(fpm_plan *p, size_t image_bytes) {
  OnlineState *o = p->online;
  if (!o->copy) FPM_CK(cudaStreamCreateWithFlags(&o->copy, cudaStreamNonBlocking));
  for (int k = 0; k < kOnlineRing; ++k) {
    if (!o->copied[k]) FPM_CK(cudaEventCreateWithFlags(&o->copied[k], cudaEventDisableTiming));
    if (!o->freed[k]) FPM_CK(cudaEventCreateWithFlags(&o->freed[k], cudaEventDisableTiming));
  }
  if (o->staging_bytes < image_bytes) {
    for (int k = 0; k < kOnlineRing; ++k) {
      if (o->staging[k]) {
        cudaEventSynchronize(o->freed[k]);
        cudaFree(o->staging[k]);
        o->staging[k] = nullptr;
      }
    }
    o->staging_bytes = 0;
    for (int k = 0; k < kOnlineRing; ++k)
      if (cudaMalloc(&o->staging[k], image_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(FPM_ENOMEM, "online staging buffers (%zu bytes each) could not be allocated", image_bytes);
      }
    o->staging_bytes = image_bytes;
  }
  return FPM_OK;
}

void online_progress(const fpm_plan *p, int32_t *launched, int32_t *total) {
  const OnlineState *o = p->online;
  *launched = o ? o->launched : 0;
  *total = o ? (int32_t)o->need.size() : 0;
}

// Launch every wave step whose LEDs have all arrived.
static int online_advance(fpm_plan *p, cudaStream_t st) {
  OnlineState *o = p->online;
  int32_t s1 = o->launched;
  while (s1 < (int32_t)o->need.size() && o->need[s1] <= o->prefix) ++s1;
  if (s1 == o->launched) return FPM_OK;
  if (o->tail && o->launched == o->tail_from && s1 == (int32_t)o->need.size()) {
    FPM_CK(cudaGraphLaunch(o->tail, st));
    o->launched = s1;
    return FPM_OK;
  }
  const int rc = enqueue_wave_steps(p, o->iters, o->launched, s1, st);
  if (rc == FPM_OK) o->launched = s1;
  return rc;
}

}  // namespace fpm

using fpm::fail;

extern "C" {

int fpm_online_begin(fpm_plan *p, int32_t iters, int32_t dtype, float counts_per_unit, void *stream) {
  fpm::clear_error();
  if (!p) return fail(FPM_EINVAL, "fpm_online_begin: null plan");
  if (p->busy) return fail(FPM_EBUSY, "plan is owned by a server job");
  if (iters < 1 || iters > p->iters) return fail(FPM_EINVAL, "iters %d outside 1..%d", iters, p->iters);
  if (dtype != FPM_U16 && dtype != FPM_F32) return fail(FPM_EINVAL, "unknown image dtype %d", dtype);
  if (!(counts_per_unit > 0) || !std::isfinite(counts_per_unit))
    return fail(FPM_EINVAL, "counts_per_unit must be positive and finite");
  cudaStream_t st = (cudaStream_t)stream;
  int rc;
  if ((rc = fpm::ensure_device_state(p))) return rc;
  if (!p->online) p->online = new fpm::OnlineState();
  fpm::OnlineState *o = p->online;
  const size_t es = dtype == FPM_U16 ? 2 : 4;
  if ((rc = fpm::online_resources(p, (size_t)p->sensor_h * p->sensor_w * es))) return rc;
  if ((rc = fpm::ensure_images(p, dtype))) return rc;
  if ((rc = fpm::begin_load(p, dtype, counts_per_unit, st))) return rc;
  o->iters = iters;
  o->dtype = dtype;
  o->pos.assign(p->n_leds, 0);
  for (int k = 0; k < p->n_leds; ++k) o->pos[p->order[k]] = k;
  o->arrived.assign(p->n_leds, 0);
  o->prefix = 0;
  o->launched = 0;
  o->pushes = 0;
  const fpm::StepLists &sl = fpm::step_lists(p, iters);
  o->need.assign(sl.n_steps, 0);
  int32_t run = 1;                         // every step needs the first LED (initial guess)
  for (int s = 0; s < sl.n_steps; ++s) {
    for (int64_t i = sl.step_off[s]; i < sl.step_off[s + 1]; ++i)
      run = std::max(run, o->pos[sl.items[i * 4 + 1]] + 1);
    o->need[s] = run;
  }
  // in LED order the last image releases every step that needs all of them
  if (o->tail) {
    cudaGraphExecDestroy(o->tail);
    o->tail = nullptr;
  }
  o->tail_from = (int32_t)(std::lower_bound(o->need.begin(), o->need.end(), p->n_leds) - o->need.begin());
  if (o->tail_from < sl.n_steps &&
      (rc = fpm::capture_wave_steps(p, iters, o->tail_from, sl.n_steps, 8, &o->tail)))
    return rc;
  o->active = true;
  return FPM_OK;
}

int fpm_online_push(fpm_plan *p, int32_t led, const void *image, int32_t on_device, int64_t stride_row,
                    void *stream) {
  fpm::clear_error();
  if (!p || !image) return fail(FPM_EINVAL, "fpm_online_push: null argument");
  fpm::OnlineState *o = p->online;
  if (!o || !o->active) return fail(FPM_ESTATE, "fpm_online_push outside fpm_online_begin .. fpm_online_finish");
  if (led < 0 || led >= p->n_leds) return fail(FPM_EINVAL, "LED %d out of range", led);
  if (o->arrived[led]) return fail(FPM_EINVAL, "LED %d was already pushed", led);
  if (stride_row < p->sensor_w) return fail(FPM_EINVAL, "stride_row %lld below the sensor width", (long long)stride_row);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = o->dtype == FPM_U16 ? 2 : 4;
  const size_t row = (size_t)p->sensor_w * es;
  const void *plane = image;
  long long pitch = stride_row;
  int k = -1;
  if (!on_device) {
    k = (int)(o->pushes % fpm::kOnlineRing);
    if (o->used[k]) FPM_CK(cudaStreamWaitEvent(o->copy, o->freed[k], 0));
    FPM_CK(cudaMemcpy2DAsync(o->staging[k], row, image, (size_t)stride_row * es, row, p->sensor_h,
                             cudaMemcpyHostToDevice, o->copy));
    FPM_CK(cudaEventRecord(o->copied[k], o->copy));
    FPM_CK(cudaStreamWaitEvent(st, o->copied[k], 0));
    plane = o->staging[k];
    pitch = p->sensor_w;
  }
  int rc = fpm::gather_tile_images(p, plane, o->dtype, 0, pitch, led, 1, st);
  if (!rc && o->pos[led] == 0) rc = fpm::run_init(p, plane, pitch, st);
  if (k >= 0) {
    if (cudaEventRecord(o->freed[k], st) != cudaSuccess && !rc) rc = fail(FPM_ECUDA, "online event");
    o->used[k] = true;
  }
  if (rc) return rc;
  o->arrived[led] = 1;
  ++o->pushes;
  while (o->prefix < p->n_leds && o->arrived[p->order[o->prefix]]) ++o->prefix;
  return fpm::online_advance(p, st);
}

int fpm_online_finish(fpm_plan *p, void *stream) {
  fpm::clear_error();
  if (!p) return fail(FPM_EINVAL, "fpm_online_finish: null plan");
  fpm::OnlineState *o = p->online;
  if (!o || !o->active) return fail(FPM_ESTATE, "fpm_online_finish without fpm_online_begin");
  if (o->prefix < p->n_leds)
    return fail(FPM_ESTATE, "%d of %d images not pushed", p->n_leds - (int)o->pushes, p->n_leds);
  const int rc = fpm::online_advance(p, (cudaStream_t)stream);
  if (rc) return rc;
  o->active = false;
  fpm::mark_loaded(p);
  return FPM_OK;
}

}  // extern "C"
