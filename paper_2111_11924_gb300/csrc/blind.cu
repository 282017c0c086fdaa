// Instantiations and launcher of the fused blinded CRT decryption
// (modexp_blind.cuh): one geometry per prime limb count, the CRT default.
#include "modexp_blind.cuh"
#include "modexp_kernels.cuh"

namespace pmk {
namespace {

struct BlindEntry {
  int limbs, tpi, threads;
  const void *fn;
  size_t smem;
};

template <int S, int TPI, int FORM, int NT = dev::kThreads>
BlindEntry make_blind() {
  return BlindEntry{S, TPI, NT, reinterpret_cast<const void *>(&dev::k_blind_crt<S, TPI, FORM, NT>),
                    dev::modexp_smem_bytes<S>(TPI, NT)};
}

// Throughput geometries (the CRT defaults), then geometries with more lanes
// per instance for small batches (a shorter chain per exponentiation).
const BlindEntry *blind_entries(int *count) {
  using dev::kChain;
  using dev::kCols;
  static const BlindEntry entries[] = {
      make_blind<2, 2, kChain>(),  make_blind<4, 2, kChain>(),  make_blind<8, 2, kChain>(),
      make_blind<16, 2, kChain>(), make_blind<32, 4, kCols, 64>(), make_blind<48, 8, kChain>(),
      make_blind<64, 8, kChain>(), make_blind<96, 8, kChain>(),  make_blind<128, 16, kChain>(),
  };
  *count = (int)(sizeof(entries) / sizeof(entries[0]));
  return entries;
}

const BlindEntry *blind_entries_latency(int *count) {
  using dev::kChain;
  static const BlindEntry entries[] = {
      make_blind<16, 8, kChain>(),  make_blind<32, 16, kChain>(), make_blind<48, 16, kChain>(),
      make_blind<64, 32, kChain>(), make_blind<96, 16, kChain>(), make_blind<128, 32, kChain>(),
  };
  *count = (int)(sizeof(entries) / sizeof(entries[0]));
  return entries;
}

}  // namespace

bool blind_crt_built(uint32_t prime_limbs) {
  int cnt = 0;
  const BlindEntry *list = blind_entries(&cnt);
  for (int i = 0; i < cnt; i++)
    if (list[i].limbs == (int)prime_limbs) return true;
  return false;
}

int launch_blind_crt(uint32_t prime_limbs, uint32_t parts, const KeyDev *keys, uint32_t K, const uint32_t *cstar,
                     const uint32_t *cr, uint32_t *out, size_t n, cudaStream_t st, uint32_t *status) {
  if (n == 0) return PMK_OK;
  if (parts < 2 || parts > (uint32_t)kMaxPrimes || (unsigned long long)K * parts > 65535ull) return PMK_EINVAL;
  int cnt = 0, dev = 0, sms = 0;
  const BlindEntry *list = blind_entries(&cnt), *e = nullptr;
  for (int i = 0; i < cnt; i++)
    if (list[i].limbs == (int)prime_limbs) e = &list[i];
  if (!e) return PMK_EUNSUPPORTED;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PMK_ECUDA;
  if ((long long)n * parts < 16LL * sms) {  // too few exponentiations to fill the GPU: shorten each one
    const BlindEntry *lat = blind_entries_latency(&cnt);
    for (int i = 0; i < cnt; i++)
      if (lat[i].limbs == (int)prime_limbs) e = &lat[i];
  }
  int rc = configure_smem(e->fn, e->smem);
  if (rc != PMK_OK) return rc;
  const long long per_key = ((long long)n + K - 1) / K;
  const int ipb = e->threads / e->tpi;
  dim3 grid((unsigned)((per_key + ipb - 1) / ipb), parts * K);
  long long nl = (long long)n;
  int np = (int)parts;
  void *args[] = {(void *)&keys, (void *)&K, (void *)&cstar, (void *)&cr, (void *)&out, (void *)&nl, (void *)&np,
                  (void *)&status};
  return cudaLaunchKernel(e->fn, grid, dim3(e->threads), args, e->smem, st) == cudaSuccess ? PMK_OK : PMK_ECUDA;
}

}  // namespace pmk
