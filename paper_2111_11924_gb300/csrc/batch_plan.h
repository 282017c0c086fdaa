// Task planning of the batched path (pmk_batch_create), free of device
// calls: which jobs get their own grid launch, and the persistent-kernel
// tasks of the others, grouped by exponentiation width and mode.
#pragma once

#include <functional>
#include <vector>

#include "pmk_internal.h"

namespace pmk {

// One job as the planner sees it.
struct PlanJob {
  const KeyDev *keys;  // the key set's K device key views
  uint32_t K, nbits, nprimes;
  int op;  // PMK_OP_ENCRYPT, PMK_OP_DECRYPT or PMK_OP_DECRYPT_CRT
  size_t n_chunks;
  const uint32_t *in;
  uint32_t *out;
};

// The tasks of one (width, mode) group, for one persistent kernel.
struct PlanGroup {
  uint32_t limbs = 0;
  bool crt = false;
  KernelConfig cfg;
  std::vector<BatchTask> tasks;
};

// A job that runs as its own grid launch.
struct PlanDirect {
  size_t job;  // index into the job list
  uint32_t limbs;
  KernelConfig cfg;
};

// Which jobs run as their own plain grid launch inside the graph (the kernel
// of pmk_*_chunks, on a stream of its own) instead of sharing a persistent
// queue:
//   - every job, when the batch holds at most kDirectMaxJobs jobs with
//     chunks: the grid kernel runs each exponentiation faster than the
//     persistent one (up to 20% on jobs too small to fill the GPU), and the
//     concurrent launches overlap as well as the shared queue does (mixed
//     64-message batch 535 vs 552 ms, 256 jobs of 1-16 chunks 61.8 vs
//     63.8 ms);
//   - in larger batches, the jobs with at least kDirectWaves GPU-fulls of
//     exponentiations: one launch per tiny job leaves most of each block's
//     shared memory unused, and 1,024 jobs of 1-8 chunks took 171 ms as
//     launches against 94 ms through the queues.
// (kDirectMaxJobs, the default limit, is defined with the context in
// pmk_internal.h.)
constexpr long long kDirectWaves = 1;

// config(limbs, crt, &cfg): the geometry for that width and mode (false if
// none); resident(limbs, cfg, crt): the exponentiations the whole GPU holds
// at once in it; direct_max_jobs: the batch size up to which every job runs
// as its own launch (kDirectMaxJobs in the library).  Jobs with no chunks
// are skipped.  A task holds up to
// 32 / TPI chunks of one key (first, first + K, ...) and, for CRT, one
// prime.  On return the groups are non-empty, widest first, with
// decryptions before encryptions inside each.  Returns PMK_OK, or
// PMK_EUNSUPPORTED when a width has no geometry or no resident capacity.
int plan_batch(const std::vector<PlanJob> &jobs, const std::function<bool(uint32_t, bool, KernelConfig *)> &config,
               const std::function<long long(uint32_t, const KernelConfig &, bool)> &resident,
               size_t direct_max_jobs, std::vector<PlanGroup> &groups, std::vector<PlanDirect> &direct);

}  // namespace pmk
