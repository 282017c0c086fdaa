// Task planning of the batched path; see batch_plan.h.
#include "batch_plan.h"

#include <algorithm>

namespace pmk {

int plan_batch(const std::vector<PlanJob> &jobs, const std::function<bool(uint32_t, bool, KernelConfig *)> &config,
               const std::function<long long(uint32_t, const KernelConfig &, bool)> &resident,
               size_t direct_max_jobs, std::vector<PlanGroup> &groups, std::vector<PlanDirect> &direct) {
  groups.clear();
  direct.clear();
  const size_t busy = (size_t)std::count_if(jobs.begin(), jobs.end(), [](const PlanJob &j) { return j.n_chunks > 0; });
  const bool all_direct = busy <= direct_max_jobs;
  auto group_for = [&](uint32_t limbs, bool crt) -> PlanGroup * {
    for (PlanGroup &g : groups)
      if (g.limbs == limbs && g.crt == crt) return &g;
    PlanGroup g;
    g.limbs = limbs;
    g.crt = crt;
    if (!config(limbs, crt, &g.cfg) || g.cfg.tpi == 0 || 32 % g.cfg.tpi) return nullptr;
    groups.push_back(g);
    return &groups.back();
  };
  for (size_t j = 0; j < jobs.size(); j++) {
    const PlanJob &jb = jobs[j];
    if (jb.n_chunks == 0) continue;
    const bool crt = jb.op == PMK_OP_DECRYPT_CRT;
    const uint32_t S = jb.nbits / 32, limbs = crt ? S / jb.nprimes : S;
    PlanGroup *g = group_for(limbs, crt);
    if (!g) return PMK_EUNSUPPORTED;
    const long long wave = resident(limbs, g->cfg, crt);  // one GPU-full
    if (wave <= 0) return PMK_EUNSUPPORTED;
    const long long instances = (long long)jb.n_chunks * (crt ? jb.nprimes : 1);
    if (all_direct || instances >= kDirectWaves * wave) {
      direct.push_back(PlanDirect{j, limbs, g->cfg});
      continue;
    }
    const uint32_t ipw = 32 / g->cfg.tpi;
    for (uint32_t k = 0; k < jb.K && k < jb.n_chunks; k++) {
      const long long count = ((long long)jb.n_chunks - k + jb.K - 1) / jb.K;
      for (long long i0 = 0; i0 < count; i0 += ipw)
        for (int prime = 0; prime < (crt ? (int)jb.nprimes : 1); prime++) {
          BatchTask t;
          t.key = jb.keys + k;
          t.in = jb.in;
          t.out = jb.out;
          t.first = k + i0 * jb.K;
          t.stride = jb.K;
          t.count = (int)std::min<long long>(ipw, count - i0);
          t.mode = crt ? 2 + prime : (jb.op == PMK_OP_ENCRYPT ? 0 : 1);
          g->tasks.push_back(t);
        }
    }
  }
  // longest work first: decryptions before encryptions within a group,
  // widest groups launched first
  for (PlanGroup &g : groups)
    std::stable_sort(g.tasks.begin(), g.tasks.end(),
                     [](const BatchTask &x, const BatchTask &y) { return (x.mode != 0) > (y.mode != 0); });
  std::stable_sort(groups.begin(), groups.end(), [](const PlanGroup &x, const PlanGroup &y) {
    return x.limbs * (x.crt ? 1 : 2) > y.limbs * (y.crt ? 1 : 2);
  });
  groups.erase(std::remove_if(groups.begin(), groups.end(), [](const PlanGroup &g) { return g.tasks.empty(); }),
               groups.end());
  return PMK_OK;
}

}  // namespace pmk
