// Serving: continuous batching of reconstruction jobs on one device.
//
// A worker thread owns the device work.  Jobs are admitted first-come
// first-served while the device memory of the admitted jobs stays within the
// budget; an admitted job's images are loaded (and its initial guess built) on
// a copy stream, overlapping the running work.  The worker then runs rounds:
// each round is one persistent-kernel launch over the next chunk of wave steps
// of every loaded job, so jobs that arrive while others run join at the next
// round and their updates share the GPU with the others'.  A job's steps run in
// order whatever the rounds, so its result is the same alone and in a mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"
#include "persistent.h"
#include "runtime.h"

namespace fpm {

using Clock = std::chrono::steady_clock;

struct Job {
  fpm_job id = 0;
  fpm_plan *plan = nullptr;
  int32_t iters = 0;
  const void *stack = nullptr;     // to load at admission (null: already loaded)
  int32_t dtype = FPM_U16, on_device = 0;
  int64_t stride_led = 0, stride_row = 0;
  float counts_per_unit = 1.f;
  size_t bytes = 0;                // device memory charged to the budget
  int32_t state = FPM_JOB_QUEUED;
  Clock::time_point t_submit, t_admit, t_done;
  bool admitted = false, done = false;
  int32_t n_steps = 0, cursor = 0;
  cudaEvent_t loaded = nullptr;
};

}  // namespace fpm

struct fpm_server {
  size_t budget = 0, used = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<fpm::Job *> queued;
  std::vector<fpm::Job *> active;
  std::map<fpm_job, fpm::Job *> jobs;
  fpm_job next_id = 1;
  bool stop = false;
  std::thread worker;
  cudaStream_t st_run = nullptr, st_load = nullptr;
  fpm::QueueDev *queue = nullptr;
  unsigned *err = nullptr;
  int32_t steps_per_round = 24;
  int64_t rounds = 0;
};

namespace fpm {

static double seconds(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double>(b - a).count();
}

static void finish(fpm_server *s, Job *j, int32_t state) {
  // caller holds s->mu
  j->state = state;
  j->done = true;
  j->t_done = Clock::now();
  if (j->admitted) s->used -= j->bytes;
  j->plan->busy = 0;
}

static void worker_loop(fpm_server *s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Job *> to_load;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // admission: first come first served while the budget holds
      while (!s->stop && !s->queued.empty() && s->used + s->queued.front()->bytes <= s->budget) {
        Job *j = s->queued.front();
        s->queued.pop_front();
        j->admitted = true;
        j->state = FPM_JOB_RUNNING;
        j->t_admit = Clock::now();
        s->used += j->bytes;
        s->active.push_back(j);
        to_load.push_back(j);
      }
      if (s->stop) {
        for (Job *j : s->queued) finish(s, j, FPM_JOB_FAILED);   // cancelled
        s->queued.clear();
      }
      if (s->stop && s->active.empty()) return;
      if (s->active.empty() && to_load.empty()) {
        s->cv.wait_for(lk, std::chrono::milliseconds(50));
        continue;
      }
    }
    for (Job *j : to_load) {      // loads overlap the rounds on the copy stream
      int rc = FPM_OK;
      if (j->stack)
        rc = load_tiles(j->plan, j->stack, j->dtype, j->on_device, j->stride_led, j->stride_row, j->counts_per_unit,
                        s->st_load);
      if (rc == FPM_OK) {
        j->n_steps = schedule_steps(j->plan, j->iters);
        if (cudaEventCreateWithFlags(&j->loaded, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(j->loaded, s->st_load) != cudaSuccess)
          rc = FPM_ECUDA;
      }
      if (rc != FPM_OK) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->active.erase(std::find(s->active.begin(), s->active.end(), j));
        finish(s, j, FPM_JOB_FAILED);
      }
    }
    // one round over every loaded job
    std::vector<Job *> runnable;
    std::vector<QueueJob> qjobs;
    int dtype = -1;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (Job *j : s->active) {
        if (cudaEventQuery(j->loaded) != cudaSuccess) continue;
        const int dt = plan_image_dtype(j->plan);
        if (dtype < 0) dtype = dt;
        if (dt != dtype) continue;                  // other image type: next round
        runnable.push_back(j);
        qjobs.push_back(QueueJob{j->plan, j->iters, j->cursor, std::min(j->n_steps, j->cursor + s->steps_per_round)});
      }
    }
    cudaGetLastError();
    if (runnable.empty()) {
      std::this_thread::sleep_for(std::chrono::microseconds(200));
      continue;
    }
    int rc = refill_queue(s->queue, qjobs, s->st_run);
    if (rc == FPM_OK) rc = launch_queue(s->queue, s->err, 0, s->st_run, nullptr);
    unsigned e[2] = {0, 0};
    if (rc == FPM_OK && (cudaStreamSynchronize(s->st_run) != cudaSuccess ||
                         cudaMemcpy(e, s->err, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess))
      rc = FPM_ECUDA;
    std::lock_guard<std::mutex> lk(s->mu);
    ++s->rounds;
    for (size_t k = 0; k < runnable.size(); ++k) {
      Job *j = runnable[k];
      if (rc != FPM_OK || e[0]) {
        finish(s, j, FPM_JOB_FAILED);
      } else {
        j->cursor = qjobs[k].step_end;
        if (j->cursor >= j->n_steps) finish(s, j, FPM_JOB_DONE);
      }
    }
    s->active.erase(std::remove_if(s->active.begin(), s->active.end(), [](Job *j) { return j->done; }),
                    s->active.end());
  }
}

}  // namespace fpm

using fpm::fail;

extern "C" {

int fpm_server_create(size_t hbm_budget_bytes, fpm_server **out) {
  fpm::clear_error();
  if (!out) return fail(FPM_EINVAL, "fpm_server_create: null argument");
  *out = nullptr;
  if (hbm_budget_bytes == 0) return fail(FPM_EINVAL, "budget must be positive");
  fpm_server *s = new fpm_server();
  s->budget = hbm_budget_bytes;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st_run, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st_load, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc((void **)&s->err, 4 * sizeof(unsigned));
  if (e != cudaSuccess) {
    delete s;
    return fail(FPM_ECUDA, "server set-up: %s", cudaGetErrorString(e));
  }
  s->queue = fpm::new_queue();
  s->worker = std::thread(fpm::worker_loop, s);
  *out = s;
  return FPM_OK;
}

int fpm_submit(fpm_server *s, fpm_plan *p, int32_t iters, const void *stack, int32_t dtype, int32_t on_device,
               int64_t stride_led, int64_t stride_row, float counts_per_unit, fpm_job *out) {
  fpm::clear_error();
  if (!s || !p || !out) return fail(FPM_EINVAL, "fpm_submit: null argument");
  if (iters < 1 || iters > p->iters) return fail(FPM_EINVAL, "iters %d outside 1..%d", iters, p->iters);
  if (!fpm::persistent_fits(p->m, p->y_hi - p->y_lo + 1))
    return fail(FPM_EINVAL, "the server runs jobs in the persistent kernel, whose shared memory cannot hold tile %d "
                "with %d update rows (FPM_EPRY_UNMASKED at m = 256)", p->m, p->y_hi - p->y_lo + 1);
  size_t bytes = 0;
  if (stack) {
    size_t sb = 0;
    int rc = fpm::validate_stack(p, stack, dtype, stride_led, stride_row, counts_per_unit, &sb);
    if (rc) return rc;
    bytes = fpm::plan_device_bytes(p, dtype);
    if (!on_device) bytes += sb;      // the stack's device staging while it loads
  } else if (fpm::plan_image_dtype(p) < 0) {
    return fail(FPM_ESTATE, "plan has no images: pass a stack or call fpm_load_tiles first");
  } else {
    bytes = fpm::plan_device_bytes(p, fpm::plan_image_dtype(p));
  }
  if (bytes > s->budget)
    return fail(FPM_EBUDGET, "job needs %zu device bytes, more than the server's budget %zu", bytes, s->budget);
  std::lock_guard<std::mutex> lk(s->mu);
  if (p->busy) return fail(FPM_EBUSY, "plan already belongs to a job");
  if (s->stop) return fail(FPM_ESTATE, "server is stopping");
  fpm::Job *j = new fpm::Job();
  j->id = s->next_id++;
  j->plan = p;
  j->iters = iters;
  j->stack = stack;
  j->dtype = dtype;
  j->on_device = on_device;
  j->stride_led = stride_led;
  j->stride_row = stride_row;
  j->counts_per_unit = counts_per_unit;
  j->bytes = bytes;
  j->t_submit = fpm::Clock::now();
  p->busy = 1;
  s->jobs[j->id] = j;
  s->queued.push_back(j);
  s->cv.notify_all();
  *out = j->id;
  return FPM_OK;
}

int fpm_poll(fpm_server *s, fpm_job job, int32_t *state, double *wait_s, double *latency_s) {
  fpm::clear_error();
  if (!s || !state) return fail(FPM_EINVAL, "fpm_poll: null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job);
  if (it == s->jobs.end()) return fail(FPM_EINVAL, "unknown job %lld", (long long)job);
  const fpm::Job *j = it->second;
  *state = j->state;
  if (wait_s) *wait_s = j->admitted ? fpm::seconds(j->t_submit, j->t_admit) : 0.0;
  if (latency_s) *latency_s = j->done ? fpm::seconds(j->t_submit, j->t_done) : 0.0;
  return FPM_OK;
}

int fpm_server_destroy(fpm_server *s) {
  if (!s) return FPM_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  for (auto &kv : s->jobs) {
    if (kv.second->loaded) cudaEventDestroy(kv.second->loaded);
    kv.second->plan->busy = 0;
    delete kv.second;
  }
  fpm::free_queue(s->queue);
  if (s->err) cudaFree(s->err);
  if (s->st_run) cudaStreamDestroy(s->st_run);
  if (s->st_load) cudaStreamDestroy(s->st_load);
  delete s;
  return FPM_OK;
}

}  // extern "C"
