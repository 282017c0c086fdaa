// Autotuner: for one key set and batch size, time every compiled kernel
// geometry (lanes per instance x Montgomery form) of the exponentiation that
// the caller will run, with the full odd-power table (window bound 5) and,
// where compiled, the small one (bound 4), and keep the fastest in the
// context.  The window
// width within the bound is chosen per exponent on the host (fewest
// products); the table size trades a few more products for more resident
// instances, which only a measurement can settle.
//
// Inputs are synthetic chunks below every modulus (top limb zero), so the
// timing covers the same schedule lengths as real ciphertexts; results of
// every geometry are bit-identical, only their speed differs.
#include <algorithm>
#include <random>
#include <vector>

#include "pmk_internal.h"

extern "C" int pmk_autotune(pmk_ctx *ctx, const pmk_keyset *ks, size_t n_chunks, int mode, int reps, uint32_t *tpi,
                            uint32_t *form, float *ms) {
  pmk::TraceRange trace("pmk_autotune");
  if (!ctx || !ks || ks->device != ctx->device || n_chunks == 0 || mode < 0 || mode > 2) return PMK_EINVAL;
  const bool crt = mode == 2;
  const uint32_t S = ks->nbits / 32;
  const uint32_t limbs = crt ? S / ks->nprimes : S;
  const pmk::ExpMode em = mode == 0 ? pmk::ExpMode::kEncrypt : (crt ? pmk::ExpMode::kCrtHalf : pmk::ExpMode::kDecrypt);
  reps = std::max(1, std::min(reps, 20));
  std::vector<pmk::KernelConfig> geoms(64);
  const int ngeom = std::min(pmk::list_configs(limbs, crt, geoms.data(), 64), 64);
  if (ngeom <= 0) return PMK_EUNSUPPORTED;
  std::vector<pmk::KernelConfig> cfgs;
  for (int table : {pmk::kTableFull, pmk::kTableSmall})
    for (int c = 0; c < ngeom; c++) {
      pmk::KernelConfig k = geoms[c];
      k.table = table;
      if (table == pmk::kTableFull || pmk::modexp_small_table_built(limbs, k, crt)) cfgs.push_back(k);
    }
  const int ncfg = (int)cfgs.size();

  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return PMK_ECUDA;
  if (prev != ks->device && cudaSetDevice(ks->device) != cudaSuccess) return PMK_ECUDA;
  const size_t words = n_chunks * S;
  std::vector<uint32_t> h(words);
  std::mt19937 gen(12345);
  for (size_t i = 0; i < words; i++) h[i] = (i % S == S - 1) ? 0u : (uint32_t)gen();
  uint32_t *d_in = nullptr, *d_out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PMK_OK;
  float best_ms = 0;
  pmk::KernelConfig best;
  if (cudaMalloc(&d_in, words * 4) != cudaSuccess || cudaMalloc(&d_out, words * 4) != cudaSuccess) rc = PMK_ENOMEM;
  if (rc == PMK_OK && (cudaMemcpy(d_in, h.data(), words * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
                       cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = PMK_ECUDA;
  for (int c = 0; c < ncfg && rc == PMK_OK; c++) {
    float t_min = 0;
    for (int r = 0; r <= reps && rc == PMK_OK; r++) {  // r = 0 warms up
      cudaEventRecord(e0, 0);
      rc = pmk::launch_modexp(em, limbs, cfgs[c], ks->d_keys, ks->K, d_in, d_out, n_chunks, 0, ks->nprimes);
      cudaEventRecord(e1, 0);
      if (rc == PMK_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = PMK_ECUDA;
      float t = 0;
      cudaEventElapsedTime(&t, e0, e1);
      if (r > 0 && (r == 1 || t < t_min)) t_min = t;
    }
    if (rc == PMK_OK && (c == 0 || t_min < best_ms)) {
      best_ms = t_min;
      best = cfgs[c];
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_in);
  cudaFree(d_out);
  if (rc == PMK_OK) {
    rc = pmk_set_kernel_config(ctx, limbs, crt ? 1 : 0, best.tpi, best.form);
    if (rc == PMK_OK) rc = pmk_set_kernel_window(ctx, limbs, crt ? 1 : 0, pmk::window_of(best.table));
    if (tpi) *tpi = best.tpi;
    if (form) *form = best.form;
    if (ms) *ms = best_ms;
  }
  if (prev != ks->device) cudaSetDevice(prev);
  return rc;
}
