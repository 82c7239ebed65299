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
  int band;         // the job's support fits the band of the band-pruned update
  int pad1;
};

struct PItem {
  int job, tile, led, slot;        // tile: index into the queue's counters
  int wave, target, width, ltile;  // target: tile's completed updates once this wave is done
};

// Jobs whose arguments travel inline in the kernel parameters (constant bank):
// the update then reads them as the wave launches do, with no shared-memory
// loads that its own shared-memory stores would force the compiler to repeat.
constexpr int kInlineJobs = 16;

struct PersistArgs {
  JobArgs inl[kInlineJobs];        // the first jobs' arguments (all of them when INL)
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

// 2-CTA clusters of 384 threads, one CTA per SM, for every tile side and for
// mixed queues, twiddles read through L1 (so that a mixed queue does not reload
// them into shared memory for every update).  A queue whose jobs all have tiles of 256 runs the layout the
// wave launches run: 4-CTA clusters of 256 threads (128 registers), two CTAs
// of different clusters per SM, twiddles read through L1 and each column's
// pixels fetched one column ahead.  The persistent configurations reach the
// other CTAs' shared memory through generic pointers (DS = 0): with the queue
// loop's state around the update, the explicit shared::cluster accesses cost
// spills.
constexpr int kPC = 2, kPT = 384, kPC256 = 4, kPT256 = 256;
using P64 = UpdateCfg<64, 8, 8, 8, kPC, kPT, 1, 1, 0, 1, 0>;
using P128 = UpdateCfg<128, 16, 8, 8, kPC, kPT, 1, 1, 0, 1, 0>;
using P192 = UpdateCfg<192, 12, 16, 16, kPC, kPT, 1, 1, 0, 1, 0>;
using P256 = UpdateCfg<256, 16, 16, 16, kPC, kPT, 1, 1, 0, 1, 0>;
using P256q = UpdateCfg<256, 16, 16, 16, kPC256, kPT256, 2, 1, 0, 1, 0>;

template <int MSEL>
constexpr int persistent_threads() { return MSEL == 256 ? kPT256 : kPT; }
template <int MSEL>
constexpr int persistent_cluster() { return MSEL == 256 ? kPC256 : kPC; }
template <int MSEL>
constexpr int persistent_min_blocks() { return MSEL == 256 ? 2 : 1; }

static size_t persistent_smem(int m, int rows, int msel) {
  switch (m) {
    case 64: return P64::smem_bytes(rows);
    case 128: return P128::smem_bytes(rows);
    case 192: return P192::smem_bytes(rows);
    default: return msel == 256 ? P256q::smem_bytes(rows) : P256::smem_bytes(rows);
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
__device__ __forceinline__ unsigned load_relaxed(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned add_relaxed(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.relaxed.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Count one finished update of entry `it` on its tile; true if it completes the
// tile's wave.  The fence before orders the cluster's writes of the update (made
// visible to this thread by the update's cluster barriers) before the count; the
// fence after a completing count orders the other clusters' writes of the wave
// before the merge that follows.
__device__ __forceinline__ bool count_done(const PersistArgs &pa, const PItem &it) {
  fence_acq_rel();
  const bool last = add_relaxed(&pa.done[it.tile], 1u) + 1u == (unsigned)it.target;
  if (last) fence_acq_rel();
  return last;
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
//
// The queue work of an entry runs inside the update before it, on the thread of
// the update's hook (cluster rank 0, last warp, which has a phase-3 row fewer
// than the others): it counts the previous update done, claims the next entry,
// reads it and looks whether its dependency is met.  The update's closing
// barrier publishes the results, so in the common case (dependency met) the
// next update starts with no barrier or wait of its own.  Otherwise the leader
// takes the pending done count first (the entry may depend on the wave it
// completes), merges if it completed a wave, and waits.
// INL = 0: the jobs' arguments are read from the table in global memory (copied
// into shared memory when the job changes); 1: from the inline table in the
// kernel parameters, indexed by the entry's job; 2: one job, whose arguments are
// the inline table's first entry at a constant offset (the update then reads
// them as immediate constant-bank operands, as in the wave launches).
// ZB: the band pruning of the update for tiles of 128 and 256 (every such job's
// support fits the band; other tile sides have no band-pruned form).
template <typename Img, int MSEL, int INL, int ZB>
__global__ void __launch_bounds__(persistent_threads<MSEL>(), persistent_min_blocks<MSEL>())
    persistent_kernel(const __grid_constant__ PersistArgs pa) {
  constexpr int PC = persistent_cluster<MSEL>();
  extern __shared__ float4 smem_raw[];
  // queue state, one copy per CTA written through distributed shared memory:
  // a ring of three entries (current, next, previous, by position mod 3);
  // s_ready: the next entry's dependency was seen met; s_last: the previous
  // entry completed its tile's wave (from the hook); s_last0, s_ok: the same
  // from the leader on the waiting path
  __shared__ PItem s_item[3];
  __shared__ int s_idx[3], s_ready, s_last, s_last0, s_ok;
  // the current job's arguments, read by the update from shared memory rather
  // than through a pointer into global memory
  __shared__ UpdateArgs s_args;
  static_assert(sizeof(UpdateArgs) % 4 == 0 && sizeof(UpdateArgs) / 4 <= kPT256, "one word per thread");
  int args_job = -1;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned q = cl.block_rank();
  const bool leader = q == 0 && threadIdx.x == 0;
  // one tile side: its twiddles stay in shared memory for the whole run (the
  // first cluster barrier below orders them before any update reads them)
  if constexpr (MSEL == 64) load_twiddles<P64>(pa.jobs[0].u, reinterpret_cast<float2 *>(smem_raw));
  if constexpr (MSEL == 128) load_twiddles<P128>(pa.jobs[0].u, reinterpret_cast<float2 *>(smem_raw));
  if constexpr (MSEL == 192) load_twiddles<P192>(pa.jobs[0].u, reinterpret_cast<float2 *>(smem_raw));
  if constexpr (MSEL == 256) load_twiddles<P256q>(pa.jobs[0].u, reinterpret_cast<float2 *>(smem_raw));
  constexpr bool load_tw = MSEL == 0;   // mixed tile sides reload them per update
  // every CTA of the cluster merges its share of a completed wave; the leader
  // then releases the tile's next wave
  // after_relaxed: the update before closed with a relaxed barrier, so a cluster
  // barrier first orders this cluster's own corrections before the merge reads them
  auto merge_wave = [&](const PItem &it, bool after_relaxed) {
    if (after_relaxed) cl.sync();
    const JobArgs *mj = pa.jobs + it.job;
    if (mj->epry)
      merge_rows(const_cast<float2 *>(mj->u.pup), mj->u.dpup, it.ltile, it.width, (int)q, PC, mj->u.y_lo,
                 mj->u.rows, mj->m, mj->u.slots, mj->u.disc, threadIdx.x, blockDim.x);
    // the cluster barrier orders every thread's pupil writes before the leader's
    // fence, which orders them (cumulatively) before the release of the wave
    cl.sync();
    if (leader) {
      __threadfence();
      store_release(&pa.merged[it.tile], (unsigned)it.wave + 1u);
    }
  };
  if (leader) {
    const int idx = (int)atomicAdd(pa.next, 1u);
    const PItem it = idx < pa.n_items ? pa.items[idx] : PItem{};
    for (int r = 0; r < PC; ++r) {
      *cl.map_shared_rank(&s_idx[0], r) = idx;
      *cl.map_shared_rank(&s_item[0], r) = it;
    }
  }
  cl.sync();
  bool pending = false;   // the previous update is not counted done yet (uniform)
  bool ready = false;     // the current entry's dependency was seen met (uniform)
  bool aborted = false;   // a dependency wait ran out or another cluster aborted (uniform)
  int k = 0;
  for (;; k = (k + 1) % 3) {
    const int cur = k, nxt = (k + 1) % 3, prv = (k + 2) % 3;
    if (s_idx[cur] >= pa.n_items) break;
    if (!ready) {
      // the current entry may depend on the wave the previous update completes
      if (pending) {
        cl.sync();                         // the update's writes (its closing barrier was relaxed)
        if (leader) {
          const int last = count_done(pa, s_item[prv]) ? 1 : 0;
          for (int r = 0; r < PC; ++r) *cl.map_shared_rank(&s_last0, r) = last;
        }
        cl.sync();
        if (s_last0) merge_wave(s_item[prv], false);
        pending = false;
      }
      if (leader) {
        const unsigned want = pa.stall_test ? 0xffffffffu : (unsigned)s_item[cur].wave;
        const bool ok = wait_for(&pa.merged[s_item[cur].tile], want, &pa.err[1], pa.timeout_ns);
        if (!ok) {
          atomicOr(&pa.err[0], 1u);        // a dependency wait ran out (or another did)
          atomicExch(&pa.err[1], 1u);
        }
        for (int r = 0; r < PC; ++r) *cl.map_shared_rank(&s_ok, r) = ok ? 1 : 0;
      }
      cl.sync();
      if (!s_ok) {
        aborted = true;
        break;
      }
    }
    const int job = s_item[cur].job;
    if (INL == 0 && job != args_job) {         // uniform: every thread read the same entry
      const JobArgs *jp = pa.jobs + job;
      if (threadIdx.x < sizeof(UpdateArgs) / 4)
        reinterpret_cast<unsigned *>(&s_args)[threadIdx.x] = reinterpret_cast<const unsigned *>(&jp->u)[threadIdx.x];
      args_job = job;
      __syncthreads();
    }
    const int4 item = make_int4(s_item[cur].ltile, s_item[cur].led, s_item[cur].slot, 0);
    const bool count_prev = pending;
    unsigned h_done = 0;                   // the hook's requests, answered by its second stage
    int h_nidx = 0;
    auto hook = [&](int stage) {
      if (stage == 0) {
        // count the previous update done and claim the next entry; the answers
        // arrive while this warp does its phase-3 rows
        if (count_prev) {
          fence_acq_rel();
          h_done = add_relaxed(&pa.done[s_item[prv].tile], 1u);
        }
        h_nidx = (int)atomicAdd(pa.next, 1u);
        return;
      }
      const int last = count_prev && h_done + 1u == (unsigned)s_item[prv].target ? 1 : 0;
      if (last) fence_acq_rel();           // the wave's other writes, before this cluster merges it
      const int nidx = load_relaxed(&pa.err[1]) ? pa.n_items : h_nidx;
      const PItem nit = nidx < pa.n_items ? pa.items[nidx] : PItem{};
      int rdy = 0;
      if (nidx < pa.n_items && !pa.stall_test) {
        const unsigned mg = load_relaxed(&pa.merged[nit.tile]), ab = load_relaxed(&pa.err[1]);
        rdy = (mg >= (unsigned)nit.wave && !ab) ? 1 : 0;
        if (rdy) fence_acq_rel();          // the merge that released it, before the next update reads
      }
      for (int r = 0; r < PC; ++r) {
        *cl.map_shared_rank(&s_idx[nxt], r) = nidx;
        *cl.map_shared_rank(&s_item[nxt], r) = nit;
        *cl.map_shared_rank(&s_last, r) = last;
        *cl.map_shared_rank(&s_ready, r) = rdy;
      }
    };
    float2 *smem = reinterpret_cast<float2 *>(smem_raw);
    const UpdateArgs &ua = INL == 2 ? pa.inl[0].u : INL == 1 ? pa.inl[job].u : s_args;
    if constexpr (MSEL == 64) {
      run_update<P64, Img>(ua, item, smem, load_tw, false, hook);
    } else if constexpr (MSEL == 128) {
      run_update<WithBand<P128, ZB>, Img>(ua, item, smem, load_tw, false, hook);
    } else if constexpr (MSEL == 192) {
      run_update<P192, Img>(ua, item, smem, load_tw, false, hook);
    } else if constexpr (MSEL == 256) {
      run_update<WithBand<P256q, ZB>, Img>(ua, item, smem, load_tw, false, hook);
    } else {
      switch (INL ? pa.inl[INL == 2 ? 0 : job].m : pa.jobs[job].m) {
        case 64: run_update<P64, Img>(ua, item, smem, load_tw, false, hook); break;
        case 128: run_update<WithBand<P128, ZB>, Img>(ua, item, smem, load_tw, false, hook); break;
        case 192: run_update<P192, Img>(ua, item, smem, load_tw, false, hook); break;
        default: run_update<WithBand<P256, ZB>, Img>(ua, item, smem, load_tw, false, hook); break;
      }
    }
    // the update's closing cluster barrier published the hook's results
    if (s_last) merge_wave(s_item[prv], true);
    ready = s_ready != 0;
    pending = true;
  }
  // the last update's done count, and its wave's merge (not after an abort)
  if (pending && !aborted) {
    const int prv = (k + 2) % 3;
    cl.sync();                             // the update's writes (its closing barrier was relaxed)
    if (leader) {
      const int last = count_done(pa, s_item[prv]) ? 1 : 0;
      for (int r = 0; r < PC; ++r) *cl.map_shared_rank(&s_last0, r) = last;
    }
    cl.sync();
    if (s_last0) merge_wave(s_item[prv], false);
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
  std::vector<JobArgs> host_jobs; // the job table (the first kInlineJobs go inline)
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
    ja[j].band = plan_band_fits(p) ? 1 : 0;
    smem = std::max(smem, persistent_smem(p->m, p->y_hi - p->y_lo + 1, msel));
  }
  if (smem > 232448) return fail(FPM_EINVAL, "a job's support is too large for the persistent kernel");
  const size_t n_items = items.size() / 8;
  if ((rc = grow(&q->items, &q->cap_items, n_items))) return rc;
  if ((rc = grow(&q->jobs, &q->cap_jobs, ja.size()))) return rc;
  if ((rc = grow(&q->counters, &q->cap_tiles, 1 + 2 * (size_t)tiles))) return rc;
  if (n_items) FPM_CK(cudaMemcpyAsync(q->items, items.data(), items.size() * 4, cudaMemcpyHostToDevice, st));
  FPM_CK(cudaMemcpyAsync(q->jobs, ja.data(), ja.size() * sizeof(JobArgs), cudaMemcpyHostToDevice, st));
  q->host_jobs = ja;
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
int persistent_cluster_size(int m) { return m == 256 ? kPC256 : kPC; }
int persistent_lanes(int m) {
  switch (m) {
    case 64: return P64::TPT;
    case 128: return P128::TPT;
    case 192: return P192::TPT;
    default: return P256q::TPT;
  }
}

int launch_queue(QueueDev *q, unsigned *err, int stall_test, cudaStream_t st, int *clusters_out) {
  if (q->n_items == 0) return FPM_OK;
  FPM_CK(cudaMemsetAsync(q->counters, 0, (1 + 2 * (size_t)q->n_tiles) * 4, st));
  FPM_CK(cudaMemsetAsync(err, 0, 2 * sizeof(unsigned), st));
  PersistArgs pa{};
  for (int j = 0; j < std::min(q->n_jobs, kInlineJobs); ++j) pa.inl[j] = q->host_jobs[j];
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
  // at most kInlineJobs jobs: their arguments from the kernel parameters (one job:
  // at constant offsets)
  const int inl = q->n_jobs == 1 ? 2 : q->n_jobs <= kInlineJobs ? 1 : 0;
  // every job of tile side 128 or 256 fits the band: the band-pruned update for them
  bool band = q->n_jobs > 0;
  for (const JobArgs &j : q->host_jobs)
    if (j.m == 128 || j.m == 256) band = band && j.band;
#define FPM_PK(M, Z)                                                                                         \
  (u16 ? (inl == 2 ? (K)&persistent_kernel<uint16_t, M, 2, Z>                                                \
                   : inl ? (K)&persistent_kernel<uint16_t, M, 1, Z> : (K)&persistent_kernel<uint16_t, M, 0, Z>) \
       : (inl == 2 ? (K)&persistent_kernel<float, M, 2, Z>                                                   \
                   : inl ? (K)&persistent_kernel<float, M, 1, Z> : (K)&persistent_kernel<float, M, 0, Z>))
  switch (q->msel) {
    case 64: k = FPM_PK(64, 0); break;
    case 128: k = band ? FPM_PK(128, kBandBlocks) : FPM_PK(128, 0); break;
    case 192: k = FPM_PK(192, 0); break;
    case 256: k = band ? FPM_PK(256, kBandBlocks) : FPM_PK(256, 0); break;
    default: k = band ? FPM_PK(0, kBandBlocks) : FPM_PK(0, 0); break;
  }
#undef FPM_PK
  FPM_CK(cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)q->smem));
  cudaLaunchConfig_t cfg{};
  cfg.blockDim = dim3(persistent_block_threads(q->msel), 1, 1);
  cfg.dynamicSmemBytes = q->smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  const int pc = persistent_cluster_size(q->msel);
  attr[0].val.clusterDim.x = (unsigned)pc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3((unsigned)pc, 1, 1);
  int clusters = 0;
  FPM_CK(cudaOccupancyMaxActiveClusters(&clusters, (void *)k, &cfg));
  if (clusters < 1) return fail(FPM_EINVAL, "the persistent kernel does not fit on this device");
  clusters = std::min(clusters, std::max(1, q->n_items));
  cfg.gridDim = dim3((unsigned)(clusters * pc), 1, 1);
  FPM_CK(cudaLaunchKernelEx(&cfg, k, pa));
  if (clusters_out) *clusters_out = clusters;
  return FPM_OK;
}

}  // namespace fpm
