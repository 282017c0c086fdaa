// Batched persistent execution: plan tasks for many jobs, group them by
// exponentiation width and mode, and capture range checks, one persistent
// kernel per group (on forked streams) and CRT recombination into a CUDA
// graph that pmk_batch_launch replays.  A CRT job contributes one task per
// (chunk group, prime) and one recombination launch.  In batches of up to
// the context's direct-launch limit (kDirectMaxJobs unless set), and for
// jobs that fill the GPU in larger ones, a job skips the queue and gets its
// own grid launch in the same graph (batch_plan.h).
#include <algorithm>
#include <new>
#include <vector>

#include "batch_plan.h"
#include "pmk_internal.h"

struct pmk_batch {
  int device = 0;
  size_t n_tasks = 0;
  int n_kernels = 0;
  pmk::BatchTask *d_tasks = nullptr;
  int *d_counters = nullptr;
  cudaStream_t capture = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> events;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

// A planned group with its place in the task array and its grid size.
struct Group {
  pmk::PlanGroup plan;
  size_t offset = 0;
  int blocks = 0;
};

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool overlap(const void *a, size_t na, const void *b, size_t nb) {
  const char *x = static_cast<const char *>(a), *y = static_cast<const char *>(b);
  return x < y + nb && y < x + na;
}

// The streams and events exist only to record the graph (cross-stream waits
// become dependency edges), and the instantiated graph is independent of the
// recorded one: all of them go as soon as the graph is instantiated, so a
// batch of many jobs does not hold a stream per job for its lifetime.
void drop_capture(pmk_batch *b) {
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  for (cudaStream_t s : b->side) cudaStreamDestroy(s);
  if (b->capture) cudaStreamDestroy(b->capture);
  b->graph = nullptr;
  b->events.clear();
  b->side.clear();
  b->capture = nullptr;
}

void release(pmk_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  drop_capture(b);
  cudaFree(b->d_tasks);
  cudaFree(b->d_counters);
}

int plan_and_capture(pmk_ctx *ctx, const pmk_job *jobs, size_t n_jobs, pmk_batch *b) {
  std::vector<pmk::PlanJob> plan_jobs(n_jobs);
  for (size_t j = 0; j < n_jobs; j++) {
    const pmk_job &jb = jobs[j];
    plan_jobs[j] = pmk::PlanJob{jb.ks->d_keys, jb.ks->K, jb.ks->nbits, jb.ks->nprimes, jb.op,
                                jb.n_chunks, jb.d_in,  jb.d_out};
  }
  auto config = [ctx](uint32_t limbs, bool crt, pmk::KernelConfig *cfg) {
    uint32_t window = 0;
    if (pmk_get_kernel_config(ctx, limbs, crt ? 1 : 0, &cfg->tpi, &cfg->form) != PMK_OK ||
        pmk_get_kernel_window(ctx, limbs, crt ? 1 : 0, &window) != PMK_OK)
      return false;
    cfg->table = window == pmk::kWindowSmall ? pmk::kTableSmall : pmk::kTableFull;
    return true;
  };
  auto resident = [](uint32_t limbs, const pmk::KernelConfig &cfg, bool crt) {
    return pmk::modexp_resident_instances(limbs, cfg, crt);
  };
  std::vector<pmk::PlanGroup> planned;
  std::vector<pmk::PlanDirect> direct;  // jobs with a grid launch of their own
  int rc = pmk::plan_batch(plan_jobs, config, resident, ctx->batch_direct_max, planned, direct);
  if (rc != PMK_OK) return rc;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) return PMK_ECUDA;
  std::vector<Group> groups(planned.size());
  std::vector<pmk::BatchTask> all;
  for (size_t gi = 0; gi < planned.size(); gi++) {
    Group &g = groups[gi];
    g.plan = std::move(planned[gi]);
    g.offset = all.size();
    all.insert(all.end(), g.plan.tasks.begin(), g.plan.tasks.end());
    const int per_sm = pmk::modexp_tasks_blocks_per_sm(g.plan.limbs, g.plan.cfg, g.plan.crt);  // raises the smem limit
    if (per_sm <= 0) return PMK_EUNSUPPORTED;
    const long long need = ((long long)g.plan.tasks.size() + 3) / 4;  // four warps per block
    g.blocks = (int)std::max<long long>(1, std::min<long long>(need, (long long)per_sm * sms));
  }
  b->n_tasks = all.size();
  b->n_kernels = (int)(groups.size() + direct.size());
  const size_t units = groups.size() + direct.size();  // one side stream per kernel
  if (!all.empty()) {
    if (cudaMalloc(&b->d_tasks, sizeof(pmk::BatchTask) * all.size()) != cudaSuccess) return PMK_ENOMEM;
    if (cudaMemcpy(b->d_tasks, all.data(), sizeof(pmk::BatchTask) * all.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return PMK_ECUDA;
  }
  if (cudaMalloc(&b->d_counters, sizeof(int) * std::max<size_t>(1, groups.size())) != cudaSuccess) return PMK_ENOMEM;
  if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess) return PMK_ECUDA;
  b->side.resize(units, nullptr);
  b->events.resize(units + 1, nullptr);
  for (auto &s : b->side)
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return PMK_ECUDA;
  for (auto &e : b->events)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return PMK_ECUDA;

  if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PMK_ECUDA;
  if (cudaMemsetAsync(b->d_counters, 0, sizeof(int) * std::max<size_t>(1, groups.size()), b->capture) != cudaSuccess)
    rc = PMK_ECUDA;
  for (size_t j = 0; j < n_jobs && rc == PMK_OK; j++)
    if (jobs[j].n_chunks)
      rc = pmk::launch_range_check(jobs[j].ks->d_keys, jobs[j].ks->K, jobs[j].ks->nbits / 32, jobs[j].d_in,
                                   jobs[j].n_chunks, ctx->d_status, b->capture);
  if (rc == PMK_OK && cudaEventRecord(b->events.back(), b->capture) != cudaSuccess) rc = PMK_ECUDA;
  for (size_t gi = 0; gi < groups.size() && rc == PMK_OK; gi++) {
    const Group &g = groups[gi];
    if (cudaStreamWaitEvent(b->side[gi], b->events.back(), 0) != cudaSuccess) {
      rc = PMK_ECUDA;
      break;
    }
    rc = pmk::launch_modexp_tasks(g.plan.limbs, g.plan.cfg, g.plan.crt, b->d_tasks + g.offset,
                                  (int)g.plan.tasks.size(), b->d_counters + gi, g.blocks, b->side[gi]);
    if (rc == PMK_OK && (cudaEventRecord(b->events[gi], b->side[gi]) != cudaSuccess ||
                         cudaStreamWaitEvent(b->capture, b->events[gi], 0) != cudaSuccess))
      rc = PMK_ECUDA;
  }
  for (size_t di = 0; di < direct.size() && rc == PMK_OK; di++) {
    const size_t u = groups.size() + di;
    const pmk_job &jb = jobs[direct[di].job];
    const pmk::ExpMode mode = jb.op == PMK_OP_ENCRYPT   ? pmk::ExpMode::kEncrypt
                              : jb.op == PMK_OP_DECRYPT ? pmk::ExpMode::kDecrypt
                                                        : pmk::ExpMode::kCrtHalf;
    if (cudaStreamWaitEvent(b->side[u], b->events.back(), 0) != cudaSuccess) {
      rc = PMK_ECUDA;
      break;
    }
    rc = pmk::launch_modexp(mode, direct[di].limbs, direct[di].cfg, jb.ks->d_keys, jb.ks->K, jb.d_in, jb.d_out,
                            jb.n_chunks, b->side[u], jb.ks->nprimes);
    if (rc == PMK_OK && (cudaEventRecord(b->events[u], b->side[u]) != cudaSuccess ||
                         cudaStreamWaitEvent(b->capture, b->events[u], 0) != cudaSuccess))
      rc = PMK_ECUDA;
  }
  for (size_t j = 0; j < n_jobs && rc == PMK_OK; j++)
    if (jobs[j].n_chunks && jobs[j].op == PMK_OP_DECRYPT_CRT) {
      const pmk_keyset *ks = jobs[j].ks;
      rc = pmk::launch_crt_sum(ks->nbits / 32, ks->nprimes, ks->d_keys, ks->K, jobs[j].d_out, jobs[j].n_chunks,
                               b->capture);
    }
  cudaGraph_t graph = nullptr;
  const cudaError_t end = cudaStreamEndCapture(b->capture, &graph);
  b->graph = graph;
  if (rc != PMK_OK) return rc;
  if (end != cudaSuccess || !graph) return PMK_ECUDA;
  if (cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) return PMK_ECUDA;
  drop_capture(b);
  return PMK_OK;
}

}  // namespace

extern "C" {

int pmk_batch_create(pmk_ctx *ctx, const pmk_job *jobs, size_t n_jobs, pmk_batch **out) {
  pmk::TraceRange trace("pmk_batch_create");
  if (!ctx || !out || (n_jobs && !jobs)) return PMK_EINVAL;
  for (size_t j = 0; j < n_jobs; j++) {
    const pmk_job &jb = jobs[j];
    if (!jb.ks || jb.ks->device != ctx->device || jb.op < 0 || jb.op > 2) return PMK_EINVAL;
    if (jb.n_chunks >= ((size_t)1 << 32)) return PMK_EINVAL;  // the per-call limit of the chunk calls
    if (jb.n_chunks == 0) continue;
    if (!jb.d_in || !jb.d_out || !aligned16(jb.d_in) || !aligned16(jb.d_out)) return PMK_EINVAL;
    const size_t bytes = jb.n_chunks * (jb.ks->nbits / 8);
    if (jb.op == PMK_OP_DECRYPT_CRT && overlap(jb.d_in, bytes, jb.d_out, bytes)) return PMK_EINVAL;
  }
  pmk_batch *b = new (std::nothrow) pmk_batch();
  if (!b) return PMK_ENOMEM;
  b->device = ctx->device;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess)) {
    delete b;
    return PMK_ECUDA;
  }
  int rc;
  try {
    rc = plan_and_capture(ctx, jobs, n_jobs, b);
  } catch (const std::bad_alloc &) {
    rc = PMK_ENOMEM;
  }
  if (rc != PMK_OK) {
    release(b);
    delete b;
  } else {
    *out = b;
  }
  if (prev != ctx->device) cudaSetDevice(prev);
  return rc;
}

int pmk_batch_launch(pmk_batch *b, void *stream) {
  pmk::TraceRange trace("pmk_batch_launch");
  if (!b || !b->exec) return PMK_EINVAL;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return PMK_ECUDA;
  if (prev != b->device && cudaSetDevice(b->device) != cudaSuccess) return PMK_ECUDA;
  const int rc = cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? PMK_OK : PMK_ECUDA;
  if (prev != b->device) cudaSetDevice(prev);
  return rc;
}

int pmk_set_batch_direct_max(pmk_ctx *ctx, size_t max_jobs) {
  pmk::TraceRange trace("pmk_set_batch_direct_max");
  if (!ctx) return PMK_EINVAL;
  ctx->batch_direct_max = max_jobs;
  return PMK_OK;
}

int pmk_batch_info(const pmk_batch *b, size_t *n_tasks, int *n_kernels) {
  if (!b) return PMK_EINVAL;
  if (n_tasks) *n_tasks = b->n_tasks;
  if (n_kernels) *n_kernels = b->n_kernels;
  return PMK_OK;
}

void pmk_batch_destroy(pmk_batch *b) {
  if (!b) return;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  release(b);
  if (prev != b->device) cudaSetDevice(prev);
  delete b;
}

}  // extern "C"
