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

// A job with at least this many GPU-fulls of exponentiations runs as one
// plain grid launch inside the graph: it fills the GPU alone, and the grid
// kernel is 3-8% faster than the persistent one on a single job of one to
// four GPU-fulls (measured from 8,000 to 28,000 2048-bit chunks), while
// mixed batches measured the same with this threshold as with four.
// Smaller jobs share the persistent queues.
constexpr long long kDirectWaves = 1;

// config(limbs, crt, &cfg): the geometry for that width and mode (false if
// none); resident(limbs, cfg, crt): the exponentiations the whole GPU holds
// at once in it.  Jobs with no chunks are skipped.  A task holds up to
// 32 / TPI chunks of one key (first, first + K, ...) and, for CRT, one
// prime.  On return the groups are non-empty, widest first, with
// decryptions before encryptions inside each.  Returns PMK_OK, or
// PMK_EUNSUPPORTED when a width has no geometry or no resident capacity.
int plan_batch(const std::vector<PlanJob> &jobs, const std::function<bool(uint32_t, bool, KernelConfig *)> &config,
               const std::function<long long(uint32_t, const KernelConfig &, bool)> &resident,
               std::vector<PlanGroup> &groups, std::vector<PlanDirect> &direct);

}  // namespace pmk
