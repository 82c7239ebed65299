// Persistent batched execution: one kernel drains a device work queue of LED
// updates taken from one or several loaded plans (tiles of different sizes
// included), in place of one launch per wave step.
//
// The queue lists the updates wave step by wave step (all jobs' step 0, then
// step 1, ...).  A cluster claims the next entry with an atomic counter, waits
// until the entry's tile has finished and merged its previous wave (Sec. 3.2:
// an update may start once the updates it depends on are done), runs the fused
// update, and counts itself done on its tile.  The cluster that completes a
// tile's wave adds the wave's pupil corrections in sequence order (both CTAs,
// 16-byte loads, every correction of a pixel pair in flight) and releases the
// next wave.  Entries are claimed in
// queue order and depend only on earlier entries, which are held by running
// clusters, so the queue cannot deadlock.  Every wait is bounded (a global
// timer); a wait that runs out sets an error code and an abort flag that ends
// the kernel, and the host reports FPM_ETIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

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

struct JobArgs {
  UpdateArgs u;     // the job's buffers; u.items unused
  int m;            // tile side
  int epry;
  int pad0, pad1;
};

struct PItem {
  int job, tile, led, slot;        // tile: index into the queue's counters
  int wave, target, width, ltile;  // target: tile's completed updates once this wave is done
};

struct PersistArgs {
  const JobArgs *jobs;
  const PItem *items;
  int n_items;
  int stall_test;                  // > 0: waits look at a flag nothing sets
  unsigned *next;                  // [1] claim counter
  unsigned *done;                  // [tiles] completed updates
  unsigned *merged;                // [tiles] waves completed and merged
  unsigned *err;                   // [0] error bits, [1] abort flag
  long long timeout_ns;
};

// 2-CTA clusters of 384 threads for every tile side; a queue whose jobs all
// have tiles of 256 runs 448 threads (14 warps, 144 registers each: the
// column phase's 128 columns per CTA then take 5 rounds of 28 transforms).
constexpr int kPC = 2, kPT = 384, kPT256 = 448;
using P64 = UpdateCfg<64, 8, 8, 8, kPC, kPT, 1>;
using P128 = UpdateCfg<128, 16, 8, 8, kPC, kPT, 1>;
using P192 = UpdateCfg<192, 12, 16, 16, kPC, kPT, 1>;
using P256 = UpdateCfg<256, 16, 16, 16, kPC, kPT, 1>;
using P256x = UpdateCfg<256, 16, 16, 16, kPC, kPT256, 1, 0>;

template <int MSEL>
constexpr int persistent_threads() { return MSEL == 256 ? kPT256 : kPT; }

static size_t persistent_smem(int m, int rows, int msel) {
  switch (m) {
    case 64: return P64::smem_bytes(rows);
    case 128: return P128::smem_bytes(rows);
    case 192: return P192::smem_bytes(rows);
    default: return msel == 256 ? P256x::smem_bytes(rows) : P256::smem_bytes(rows);
  }
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned load_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void store_release(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned add_acq_rel(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Wait until *flag >= want; false if the abort flag is raised or the time runs out.
__device__ bool wait_for(const unsigned *flag, unsigned want, const unsigned *abort_flag, long long timeout_ns) {
  const unsigned long long t0 = global_ns();
  unsigned sleep = 32;
  for (;;) {
    if (load_acquire(flag) >= want) return true;
    if (load_acquire(abort_flag)) return false;
    if ((long long)(global_ns() - t0) > timeout_ns) return false;
    __nanosleep(sleep);
    if (sleep < 2048) sleep *= 2;
  }
}

// MSEL = 0: any tile side (dispatch per entry); MSEL = m: every job has tile side m,
// so the kernel carries only that variant (and its register needs).
template <typename Img, int MSEL>
__global__ void __launch_bounds__(persistent_threads<MSEL>(), 1) persistent_kernel(const __grid_constant__ PersistArgs pa) {
  extern __shared__ float4 smem_raw[];
  // the cluster leader claims the next entry while the current one waits on its
  // dependency and hands both to the cluster through these (entries double-
  // buffered).  s_ok (dependency met) and s_last (wave completed) are separate:
  // between a read of either and the leader's next write of it lies a cluster
  // barrier inside the update.
  __shared__ int s_idx[2], s_ok, s_last;
  __shared__ PItem s_item[2];
  // the current job's arguments, read by the update from shared memory rather
  // than through a pointer into global memory
  __shared__ UpdateArgs s_args;
  static_assert(sizeof(UpdateArgs) % 4 == 0 && sizeof(UpdateArgs) / 4 <= kPT, "one word per thread");
  int args_job = -1;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned q = cl.block_rank();
  const bool leader = q == 0 && threadIdx.x == 0;
  // one tile side: its twiddles stay in shared memory for the whole run (the
  // first cluster barrier below orders them before any update reads them)
  if constexpr (MSEL == 64) load_twiddles<P64>(pa.jobs[0].u, reinterpret_cast<float2 *>(smem_raw));
  if constexpr (MSEL == 128) load_twiddles<P128>(pa.jobs[0].u, reinterpret_cast<float2 *>(smem_raw));
  if constexpr (MSEL == 192) load_twiddles<P192>(pa.jobs[0].u, reinterpret_cast<float2 *>(smem_raw));
  if constexpr (MSEL == 256) load_twiddles<P256x>(pa.jobs[0].u, reinterpret_cast<float2 *>(smem_raw));
  constexpr bool load_tw = MSEL == 0;   // mixed tile sides reload them per update
  if (leader) {
    const int idx = (int)atomicAdd(pa.next, 1u);
    const PItem it = idx < pa.n_items ? pa.items[idx] : PItem{};
    for (int r = 0; r < kPC; ++r) {
      *cl.map_shared_rank(&s_idx[0], r) = idx;
      *cl.map_shared_rank(&s_item[0], r) = it;
    }
  }
  cl.sync();
  for (int k = 0;; k ^= 1) {
    if (s_idx[k] >= pa.n_items) break;
    if (leader) {
      const PItem it = s_item[k];
      int nidx = (int)atomicAdd(pa.next, 1u);        // claim ahead; its latency overlaps the wait
      const unsigned want = pa.stall_test ? 0xffffffffu : (unsigned)it.wave;
      const bool ok = wait_for(&pa.merged[it.tile], want, &pa.err[1], pa.timeout_ns);
      if (!ok) {
        atomicOr(&pa.err[0], 1u);        // a dependency wait ran out (or another did)
        atomicExch(&pa.err[1], 1u);
      }
      if (load_acquire(&pa.err[1])) nidx = pa.n_items;
      const PItem nit = nidx < pa.n_items ? pa.items[nidx] : PItem{};
      for (int r = 0; r < kPC; ++r) {
        *cl.map_shared_rank(&s_ok, r) = ok ? 1 : 0;
        *cl.map_shared_rank(&s_idx[k ^ 1], r) = nidx;
        *cl.map_shared_rank(&s_item[k ^ 1], r) = nit;
      }
    }
    cl.sync();
    if (!s_ok) break;
    // the item is re-read from shared memory after the update, so it does not
    // stay in registers across it
    const int job = s_item[k].job;
    const JobArgs *jp = pa.jobs + job;
    if (job != args_job) {                 // uniform: every thread read the same item
      if (threadIdx.x < sizeof(UpdateArgs) / 4)
        reinterpret_cast<unsigned *>(&s_args)[threadIdx.x] = reinterpret_cast<const unsigned *>(&jp->u)[threadIdx.x];
      args_job = job;
      __syncthreads();
    }
    const int4 item = make_int4(s_item[k].ltile, s_item[k].led, s_item[k].slot, 0);
    float2 *smem = reinterpret_cast<float2 *>(smem_raw);
    if constexpr (MSEL == 64) {
      run_update<P64, Img>(s_args, item, smem, load_tw);
    } else if constexpr (MSEL == 128) {
      run_update<P128, Img>(s_args, item, smem, load_tw);
    } else if constexpr (MSEL == 192) {
      run_update<P192, Img>(s_args, item, smem, load_tw);
    } else if constexpr (MSEL == 256) {
      run_update<P256x, Img>(s_args, item, smem, load_tw);
    } else {
      switch (jp->m) {
        case 64: run_update<P64, Img>(s_args, item, smem, load_tw); break;
        case 128: run_update<P128, Img>(s_args, item, smem, load_tw); break;
        case 192: run_update<P192, Img>(s_args, item, smem, load_tw); break;
        default: run_update<P256, Img>(s_args, item, smem, load_tw); break;
      }
    }
    const PItem done_it = s_item[k];
    // run_update ends with a cluster barrier: all of this update's writes are issued
    if (leader) {
      __threadfence();
      const unsigned old = add_acq_rel(&pa.done[done_it.tile], 1u);
      const int last = (old + 1u == (unsigned)done_it.target) ? 1 : 0;
      for (int r = 0; r < kPC; ++r) *cl.map_shared_rank(&s_last, r) = last;
    }
    cl.sync();
    if (s_last) {          // this cluster completed the tile's wave: merge it, release the next
      const JobArgs *mj = pa.jobs + done_it.job;
      if (mj->epry)
        merge_rows(const_cast<float2 *>(mj->u.pup), mj->u.dpup, done_it.ltile, done_it.width, (int)q, kPC,
                   mj->u.y_lo, mj->u.rows, mj->m, mj->u.slots, mj->u.disc, threadIdx.x, blockDim.x);
      __threadfence();
      cl.sync();
      if (leader) {
        __threadfence();
        store_release(&pa.merged[done_it.tile], (unsigned)done_it.wave + 1u);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

int32_t schedule_steps(fpm_plan *p, int32_t iters) { return step_lists(p, iters).n_steps; }

int build_queue(const std::vector<QueueJob> &jobs, std::vector<int32_t> &items_out, int32_t *n_tiles_out) {
  std::vector<const StepLists *> sls;
  std::vector<int32_t> s0, s1, bases;
  int32_t span = 0, tiles = 0;
  for (const QueueJob &j : jobs) {
    const StepLists &sl = step_lists(j.plan, j.iters);
    sls.push_back(&sl);
    const int32_t b = std::max(0, j.step_begin);
    const int32_t e = j.step_end < 0 ? sl.n_steps : std::min(j.step_end, sl.n_steps);
    s0.push_back(b);
    s1.push_back(e);
    span = std::max(span, e - b);
    bases.push_back(tiles);
    tiles += j.plan->n_tiles;
  }
  items_out.clear();
  std::vector<int32_t> cum(tiles, 0);
  for (int r = 0; r < span; ++r)                 // relative step r of every job
    for (size_t jb = 0; jb < jobs.size(); ++jb) {
      const int s = s0[jb] + r;
      if (s >= s1[jb]) continue;
      const StepLists &sl = *sls[jb];
      const int64_t i0 = sl.step_off[s], i1 = sl.step_off[s + 1];
      for (int64_t k = i0; k < i1;) {            // items of a step are sorted by tile
        const int32_t t = sl.items[k * 4];
        int64_t e = k;
        while (e < i1 && sl.items[e * 4] == t) ++e;
        const int32_t w = (int32_t)(e - k);
        const int32_t gt = bases[jb] + t;
        cum[gt] += w;
        for (int64_t u = k; u < e; ++u) {
          const int32_t *it = sl.items.data() + u * 4;
          // waves are counted from the first step of this run
          const int32_t rec[8] = {(int32_t)jb, gt, it[1], it[2], r, cum[gt], w, t};
          items_out.insert(items_out.end(), rec, rec + 8);
        }
        k = e;
      }
    }
  *n_tiles_out = tiles;
  return FPM_OK;
}

struct QueueDev {
  PItem *items = nullptr;
  JobArgs *jobs = nullptr;
  unsigned *counters = nullptr;   // next, done[tiles], merged[tiles]
  size_t cap_items = 0, cap_jobs = 0, cap_tiles = 0;
  int n_items = 0, n_tiles = 0, n_jobs = 0;
  size_t smem = 0;
  int dtype = FPM_U16;
  int msel = 0;                   // common tile side of the jobs, 0 if mixed
};

void free_queue(QueueDev *q) {
  if (!q) return;
  if (q->items) cudaFree(q->items);
  if (q->jobs) cudaFree(q->jobs);
  if (q->counters) cudaFree(q->counters);
  delete q;
}

template <class T>
static int grow(T **p, size_t *cap, size_t need) {
  if (*cap >= need) return FPM_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  const size_t n = std::max<size_t>(need, 16);
  cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
  if (e != cudaSuccess) return fail(FPM_ENOMEM, "persistent queue allocation failed: %s", cudaGetErrorString(e));
  *cap = n;
  return FPM_OK;
}

int refill_queue(QueueDev *q, const std::vector<QueueJob> &jobs, cudaStream_t st) {
  if (jobs.empty()) return fail(FPM_EINVAL, "empty queue");
  std::vector<int32_t> items;
  int32_t tiles = 0;
  int rc = build_queue(jobs, items, &tiles);
  if (rc) return rc;
  const int dtype = plan_image_dtype(jobs[0].plan);
  std::vector<JobArgs> ja(jobs.size());
  size_t smem = 0;
  int msel = jobs[0].plan->m;
  for (const QueueJob &j : jobs)
    if (j.plan->m != msel) msel = 0;
  for (size_t j = 0; j < jobs.size(); ++j) {
    fpm_plan *p = jobs[j].plan;
    if (plan_image_dtype(p) != dtype) return fail(FPM_EINVAL, "jobs of one persistent run must share the image type");
    std::memset(&ja[j], 0, sizeof(JobArgs));
    ja[j].u = plan_update_args(p);
    ja[j].m = p->m;
    ja[j].epry = p->epry ? 1 : 0;
    smem = std::max(smem, persistent_smem(p->m, p->y_hi - p->y_lo + 1, msel));
  }
  if (smem > 232448) return fail(FPM_EINVAL, "a job's support is too large for the persistent kernel");
  const size_t n_items = items.size() / 8;
  if ((rc = grow(&q->items, &q->cap_items, n_items))) return rc;
  if ((rc = grow(&q->jobs, &q->cap_jobs, ja.size()))) return rc;
  if ((rc = grow(&q->counters, &q->cap_tiles, 1 + 2 * (size_t)tiles))) return rc;
  if (n_items) FPM_CK(cudaMemcpyAsync(q->items, items.data(), items.size() * 4, cudaMemcpyHostToDevice, st));
  FPM_CK(cudaMemcpyAsync(q->jobs, ja.data(), ja.size() * sizeof(JobArgs), cudaMemcpyHostToDevice, st));
  q->n_items = (int)n_items;
  q->n_tiles = tiles;
  q->n_jobs = (int)jobs.size();
  q->smem = smem;
  q->dtype = dtype;
  q->msel = msel;
  return FPM_OK;
}

QueueDev *new_queue() { return new QueueDev(); }

int make_queue(const std::vector<QueueJob> &jobs, QueueDev **out) {
  *out = nullptr;
  QueueDev *q = new QueueDev();
  int rc = refill_queue(q, jobs, nullptr);
  if (rc == FPM_OK) rc = cudaStreamSynchronize(nullptr) == cudaSuccess ? FPM_OK : fail(FPM_ECUDA, "queue upload");
  if (rc) {
    free_queue(q);
    return rc;
  }
  *out = q;
  return FPM_OK;
}

int queue_items(const QueueDev *q) { return q ? q->n_items : 0; }

int persistent_block_threads(int m) { return m == 256 ? kPT256 : kPT; }
bool persistent_fits(int m, int rows) {
  return std::max(persistent_smem(m, rows, m), persistent_smem(m, rows, 0)) <= 232448;
}
int persistent_cluster_size(int) { return kPC; }
int persistent_lanes(int m) {
  switch (m) {
    case 64: return P64::TPT;
    case 128: return P128::TPT;
    case 192: return P192::TPT;
    default: return P256x::TPT;
  }
}

int launch_queue(QueueDev *q, unsigned *err, int stall_test, cudaStream_t st, int *clusters_out) {
  if (q->n_items == 0) return FPM_OK;
  FPM_CK(cudaMemsetAsync(q->counters, 0, (1 + 2 * (size_t)q->n_tiles) * 4, st));
  FPM_CK(cudaMemsetAsync(err, 0, 2 * sizeof(unsigned), st));
  PersistArgs pa{};
  pa.jobs = q->jobs;
  pa.items = q->items;
  pa.n_items = q->n_items;
  pa.stall_test = stall_test;
  pa.next = q->counters;
  pa.done = q->counters + 1;
  pa.merged = q->counters + 1 + q->n_tiles;
  pa.err = err;
  pa.timeout_ns = stall_test ? 50000000LL : 2000000000LL;   // 50 ms for the test hook, else 2 s
  using K = void (*)(PersistArgs);
  const bool u16 = q->dtype == FPM_U16;
  K k;
  switch (q->msel) {
    case 64: k = u16 ? (K)&persistent_kernel<uint16_t, 64> : (K)&persistent_kernel<float, 64>; break;
    case 128: k = u16 ? (K)&persistent_kernel<uint16_t, 128> : (K)&persistent_kernel<float, 128>; break;
    case 192: k = u16 ? (K)&persistent_kernel<uint16_t, 192> : (K)&persistent_kernel<float, 192>; break;
    case 256: k = u16 ? (K)&persistent_kernel<uint16_t, 256> : (K)&persistent_kernel<float, 256>; break;
    default: k = u16 ? (K)&persistent_kernel<uint16_t, 0> : (K)&persistent_kernel<float, 0>; break;
  }
  FPM_CK(cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)q->smem));
  cudaLaunchConfig_t cfg{};
  cfg.blockDim = dim3(persistent_block_threads(q->msel), 1, 1);
  cfg.dynamicSmemBytes = q->smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kPC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(kPC, 1, 1);
  int clusters = 0;
  FPM_CK(cudaOccupancyMaxActiveClusters(&clusters, (void *)k, &cfg));
  if (clusters < 1) return fail(FPM_EINVAL, "the persistent kernel does not fit on this device");
  clusters = std::min(clusters, std::max(1, q->n_items));
  cfg.gridDim = dim3((unsigned)(clusters * kPC), 1, 1);
  FPM_CK(cudaLaunchKernelEx(&cfg, k, pa));
  if (clusters_out) *clusters_out = clusters;
  return FPM_OK;
}

}  // namespace fpm
