// Host interface of the persistent batched kernel (persistent.cu).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "internal.h"

namespace fpm {

// One job of a persistent run: a loaded plan, how many loops of its schedule,
// and which of that schedule's wave steps this run covers ([step_begin,
// step_end); step_end < 0 means to the end).  Runs over consecutive step
// ranges compute exactly what one run over all steps computes.
struct QueueJob {
  fpm_plan *plan;
  int32_t iters;
  int32_t step_begin = 0;
  int32_t step_end = -1;
};

struct QueueDev;   // device work queue, job table and counters

// Flatten the jobs' wave steps into one queue (step-major, so that every
// entry depends only on earlier ones): 8 ints per entry.
int build_queue(const std::vector<QueueJob> &jobs, std::vector<int32_t> &items_out, int32_t *n_tiles_out);
// An empty queue whose buffers grow on the first refill.
QueueDev *new_queue();
// Build and upload the queue of `jobs` (all loaded, same image type).
int make_queue(const std::vector<QueueJob> &jobs, QueueDev **out);
// Rebuild an existing queue for new jobs, reusing its device buffers when they
// are large enough (stream-ordered uploads on `st`).
int refill_queue(QueueDev *q, const std::vector<QueueJob> &jobs, cudaStream_t st);
void free_queue(QueueDev *q);
// Number of wave steps of a plan's schedule of `iters` loops.
int32_t schedule_steps(fpm_plan *p, int32_t iters);
int queue_items(const QueueDev *q);
// Threads per CTA of the persistent kernel for a queue whose jobs all have tile side m (0: mixed).
int persistent_block_threads(int m);
// Whether tiles of side m with `rows` support rows fit the persistent kernel's shared
// memory, in a queue of that side alone and in a mixed one.
bool persistent_fits(int m, int rows);
// CTAs per cluster of the persistent kernel for a queue whose jobs all have tile side m (0: mixed).
int persistent_cluster_size(int m);
// Lanes per 1-D transform of the persistent kernel's update for tile side m.
int persistent_lanes(int m);
// Reset the counters and `err` ([0] error bits, [1] abort flag) and launch the
// persistent kernel on `st`.  stall_test > 0 makes every dependency wait look
// at a flag nothing sets, with a 50 ms limit (exercises the timeout path).
int launch_queue(QueueDev *q, unsigned *err, int stall_test, cudaStream_t st, int *clusters_out);

}  // namespace fpm
