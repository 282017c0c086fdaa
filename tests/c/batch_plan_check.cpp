// Host check of the batch planner (batch_plan.cpp) with stand-in geometry
// and capacity functions; no GPU.  For random mixes of jobs (widths, key
// counts, prime counts, operations, sizes from 0 to several GPU-fulls) it
// checks that:
//   - a job goes to its own grid launch exactly when the batch holds at most
//     direct_max_jobs jobs with chunks (drawn at random around the trial's
//     job count, so both rules are exercised) or its exponentiations reach
//     kDirectWaves GPU-fulls; every other job's chunks (and, for CRT, every
//     prime of every chunk) are covered by exactly one task;
//   - a task holds 1 .. 32 / TPI chunks of one key (first = key mod K,
//     stride K), the job's buffers, and the job's mode;
//   - groups are non-empty and distinct per (width, mode), carry the
//     geometry of their width, come widest first, and hold decryptions
//     before encryptions;
//   - a width without a geometry or without capacity is refused.
#include <cstdint>
#include <cstdio>
#include <map>
#include <set>
#include <tuple>
#include <vector>

#include "batch_plan.h"

namespace {

uint64_t g_state = 0x50444D4B42415443ull;
uint32_t rnd(uint32_t n) {  // xorshift64*, uniform enough below n
  g_state ^= g_state >> 12;
  g_state ^= g_state << 25;
  g_state ^= g_state >> 27;
  return (uint32_t)(((g_state * 0x2545F4914F6CDD1Dull) >> 32) % n);
}

int g_failures = 0, g_checks = 0;
void expect(bool ok, const char *what, int trial) {
  g_checks++;
  if (!ok && g_failures++ < 20) std::printf("FAIL %s (trial %d)\n", what, trial);
}

// Stand-in geometry: lanes per instance by width, as the built-in defaults.
bool config(uint32_t limbs, bool crt, pmk::KernelConfig *cfg) {
  static const std::map<uint32_t, uint32_t> tpi = {{16, 2}, {32, 4}, {48, 8}, {64, 8}, {96, 8}, {128, 16}};
  auto it = tpi.find(limbs);
  if (it == tpi.end()) return false;
  cfg->tpi = it->second;
  cfg->form = crt ? 1 : 0;
  cfg->table = pmk::kTableFull;
  return true;
}
long long resident(uint32_t limbs, const pmk::KernelConfig &cfg, bool) { return 152LL * 3 * (128 / cfg.tpi) + limbs; }

void trial(int t) {
  const uint32_t widths[] = {1024, 2048, 3072, 4096};
  const int njobs = 1 + (int)rnd(12);
  std::vector<pmk::PlanJob> jobs;
  std::vector<std::vector<pmk::KeyDev>> keys(njobs);  // stand-in key views (never dereferenced)
  std::vector<std::vector<uint32_t>> bufs(2 * njobs, std::vector<uint32_t>(1));
  for (int j = 0; j < njobs; j++) {
    pmk::PlanJob jb;
    jb.nbits = widths[rnd(4)];
    jb.nprimes = 2;
    if (jb.nbits == 3072 && rnd(2)) jb.nprimes = 3;
    if (jb.nbits == 4096 && rnd(2)) jb.nprimes = 4;
    jb.K = 1 + rnd(20);
    keys[j].resize(jb.K);
    jb.keys = keys[j].data();
    jb.op = (int)rnd(3);
    const uint32_t pick = rnd(10);
    jb.n_chunks = pick == 0 ? 0 : pick < 7 ? rnd(3000) : 20000 + rnd(200000);
    jb.in = bufs[2 * j].data();
    jb.out = bufs[2 * j + 1].data();
    jobs.push_back(jb);
  }
  size_t busy = 0;
  for (const auto &jb : jobs) busy += jb.n_chunks > 0;
  const uint32_t pick_max = rnd(4);
  const size_t direct_max_jobs = pick_max == 0 ? 0 : pick_max == 1 ? (busy ? busy - 1 : 0) : pick_max == 2 ? busy
                                                                                                        : pmk::kDirectMaxJobs;
  const bool all_direct = busy <= direct_max_jobs;
  std::vector<pmk::PlanGroup> groups;
  std::vector<pmk::PlanDirect> direct;
  const int rc = pmk::plan_batch(jobs, config, resident, direct_max_jobs, groups, direct);
  expect(rc == PMK_OK, "planning succeeds", t);
  if (rc != PMK_OK) return;

  std::set<size_t> direct_jobs;
  for (const auto &d : direct) direct_jobs.insert(d.job);
  expect(direct_jobs.size() == direct.size(), "one grid launch per direct job", t);
  // coverage: (job, chunk, prime) -> times covered
  std::map<std::tuple<size_t, long long, int>, int> cover;
  std::set<std::pair<uint32_t, bool>> seen_groups;
  long long prev_key = -1;
  for (const auto &g : groups) {
    expect(!g.tasks.empty(), "no empty group", t);
    expect(seen_groups.insert({g.limbs, g.crt}).second, "one group per (width, mode)", t);
    pmk::KernelConfig want;
    expect(config(g.limbs, g.crt, &want) && want.tpi == g.cfg.tpi, "group geometry", t);
    const long long key = (long long)g.limbs * (g.crt ? 1 : 2);
    expect(prev_key < 0 || key <= prev_key, "widest group first", t);
    prev_key = key;
    bool seen_encrypt = false;
    for (const auto &task : g.tasks) {
      if (task.mode == 0) seen_encrypt = true;
      expect(!(seen_encrypt && task.mode != 0), "decryptions before encryptions", t);
      size_t j = 0;
      while (j < jobs.size() && jobs[j].in != task.in) j++;
      expect(j < jobs.size(), "task points at a job", t);
      if (j == jobs.size()) continue;
      const pmk::PlanJob &jb = jobs[j];
      expect(task.out == jb.out, "task output buffer", t);
      expect(!direct_jobs.count(j), "no tasks for a direct job", t);
      const bool crt = jb.op == PMK_OP_DECRYPT_CRT;
      expect(g.crt == crt && g.limbs == (crt ? jb.nbits / 32 / jb.nprimes : jb.nbits / 32), "task in its group", t);
      const int want_mode = jb.op == PMK_OP_ENCRYPT ? 0 : 1;
      expect(crt ? (task.mode >= 2 && task.mode < 2 + (int)jb.nprimes) : task.mode == want_mode, "task mode", t);
      expect(task.count >= 1 && task.count <= (int)(32 / g.cfg.tpi), "chunks per task", t);
      expect(task.stride == jb.K && task.first >= 0 && task.key == jb.keys + task.first % jb.K, "task key", t);
      for (int i = 0; i < task.count; i++) {
        const long long c = task.first + (long long)i * task.stride;
        expect(c < (long long)jb.n_chunks, "task chunk in range", t);
        cover[{j, c, crt ? task.mode - 2 : 0}]++;
      }
    }
  }
  for (size_t j = 0; j < jobs.size(); j++) {
    const pmk::PlanJob &jb = jobs[j];
    const bool crt = jb.op == PMK_OP_DECRYPT_CRT;
    const uint32_t limbs = crt ? jb.nbits / 32 / jb.nprimes : jb.nbits / 32;
    pmk::KernelConfig cfg;
    config(limbs, crt, &cfg);
    const long long instances = (long long)jb.n_chunks * (crt ? jb.nprimes : 1);
    const bool big = jb.n_chunks && (all_direct || instances >= pmk::kDirectWaves * resident(limbs, cfg, crt));
    expect(big == (direct_jobs.count(j) == 1), "grid launch exactly for small batches and jobs of a GPU-full", t);
    if (big || jb.n_chunks == 0) continue;
    for (long long c = 0; c < (long long)jb.n_chunks; c++)
      for (int p = 0; p < (crt ? (int)jb.nprimes : 1); p++) {
        auto it = cover.find({j, c, p});
        expect(it != cover.end() && it->second == 1, "every chunk and prime exactly once", t);
      }
  }
}

}  // namespace

int main() {
  for (int t = 0; t < 300; t++) trial(t);
  // refusals: a width with no geometry, a geometry with no capacity
  std::vector<pmk::KeyDev> kd(2);
  std::vector<uint32_t> in(1), out(1);
  std::vector<pmk::PlanJob> odd = {pmk::PlanJob{kd.data(), 2, 1280, 2, PMK_OP_DECRYPT, 10, in.data(), out.data()}};
  std::vector<pmk::PlanGroup> groups;
  std::vector<pmk::PlanDirect> direct;
  expect(pmk::plan_batch(odd, config, resident, 0, groups, direct) == PMK_EUNSUPPORTED, "no geometry refused", -1);
  auto none = [](uint32_t, const pmk::KernelConfig &, bool) { return 0LL; };
  odd[0].nbits = 2048;
  expect(pmk::plan_batch(odd, config, none, 0, groups, direct) == PMK_EUNSUPPORTED, "no capacity refused", -1);
  std::printf("%d checks, %d failures\n", g_checks, g_failures);
  return g_failures ? 1 : 0;
}
