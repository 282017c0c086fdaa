// C ABI of the PMKRSA library (include/pmkrsa.h): argument checks, key-set
// upload, and the order of kernel launches for each call.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>

#include "pmk_internal.h"

namespace {

using pmk::HostKey;
using pmk::KeyDev;

// Makes the context's device current for the duration of a call.
class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    ok_ = cudaGetDevice(&prev_) == cudaSuccess && (prev_ == dev || cudaSetDevice(dev) == cudaSuccess);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (ok_ && cudaGetDevice(&cur) == cudaSuccess && cur != prev_) cudaSetDevice(prev_);
  }
  bool ok() const { return ok_; }

 private:
  int prev_ = 0;
  bool ok_ = false;
};

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool overlap(const void *a, size_t na, const void *b, size_t nb) {
  const char *x = static_cast<const char *>(a), *y = static_cast<const char *>(b);
  return x < y + nb && y < x + na;
}

// Make the staging buffer hold at least `bytes` for work enqueued on `st`:
// first order `st` after the buffer's last use (on whatever stream), then
// grow it in stream order if it is too small.  Pair with release().
int acquire(pmk::Staging &s, size_t bytes, cudaStream_t st) {
  if (!s.last_use && cudaEventCreateWithFlags(&s.last_use, cudaEventDisableTiming) != cudaSuccess) return PMK_ECUDA;
  if (cudaStreamWaitEvent(st, s.last_use, 0) != cudaSuccess) return PMK_ECUDA;
  if (s.cap >= bytes) return PMK_OK;
  if (s.ptr && cudaFreeAsync(s.ptr, st) != cudaSuccess) return PMK_ECUDA;
  s.ptr = nullptr;
  s.cap = 0;
  if (cudaMallocAsync(&s.ptr, bytes, st) != cudaSuccess) {
    s.ptr = nullptr;
    return PMK_ENOMEM;
  }
  s.cap = bytes;
  return PMK_OK;
}

// Mark the end of this call's use of the buffer: everything enqueued on `st`
// so far.
void release(pmk::Staging &s, cudaStream_t st) {
  if (s.last_use) cudaEventRecord(s.last_use, st);
}

// Wait for the buffer's last use, then free it and its event.
void drop(pmk::Staging &s) {
  if (s.last_use) cudaEventSynchronize(s.last_use);
  if (s.ptr) {
    cudaFreeAsync(s.ptr, nullptr);
    cudaStreamSynchronize(nullptr);
  }
  if (s.last_use) cudaEventDestroy(s.last_use);
  s = pmk::Staging{};
}

// Kernel geometry for an exponentiation over `limbs` limbs: the context's
// override for this mode, else the built-in default.
pmk::KernelConfig cfg_for(const pmk_ctx *ctx, uint32_t limbs, bool crt) {
  const uint32_t key = limbs << 1 | (crt ? 1u : 0u);
  auto it = ctx->cfg.find(key);
  pmk::KernelConfig c = it != ctx->cfg.end() ? it->second : pmk::default_config(limbs, crt);
  // The small table applies where this geometry is compiled with it.
  auto t = ctx->table.find(key);
  const bool small = t != ctx->table.end() && t->second == pmk::kTableSmall &&
                     pmk::modexp_small_table_built(limbs, c, crt);
  c.table = small ? pmk::kTableSmall : pmk::kTableFull;
  return c;
}

// Whether any geometry for (limbs, crt) is compiled with the small table.
bool small_table_available(uint32_t limbs, bool crt) {
  pmk::KernelConfig v[64];
  const int n = std::min(pmk::list_configs(limbs, crt, v, 64), 64);
  for (int i = 0; i < n; i++)
    if (pmk::modexp_small_table_built(limbs, v[i], crt)) return true;
  return false;
}

size_t push(std::vector<uint32_t> &blob, const std::vector<uint32_t> &v) {
  while (blob.size() % 4) blob.push_back(0);  // 16-byte alignment for vector loads
  const size_t off = blob.size();
  blob.insert(blob.end(), v.begin(), v.end());
  return off;
}

int upload(pmk_keyset *ks) {
  std::vector<uint32_t> blob;
  struct Offs {
    size_t N, R2, se[2], sd[2], P[pmk::kMaxPrimes], R2h[pmk::kMaxPrimes], R3h[pmk::kMaxPrimes],
        sh[2][pmk::kMaxPrimes], shi[2][pmk::kMaxPrimes], cs[pmk::kMaxPrimes], sb[pmk::kMaxPrimes], el, dl;
  };
  std::vector<Offs> offs(ks->K);
  for (uint32_t k = 0; k < ks->K; k++) {
    const HostKey &h = ks->keys[k];
    Offs &o = offs[k];
    o.N = push(blob, h.N);
    o.R2 = push(blob, h.R2);
    for (int t = 0; t < 2; t++) {
      o.se[t] = push(blob, h.sched_e[t].steps);
      o.sd[t] = push(blob, h.sched_d[t].steps);
    }
    for (uint32_t i = 0; i < h.nprimes; i++) {
      o.P[i] = push(blob, h.pr[i]);
      o.R2h[i] = push(blob, h.R2h[i]);
      o.R3h[i] = push(blob, h.R3h[i]);
      for (int t = 0; t < 2; t++) {
        o.sh[t][i] = push(blob, h.sched_h[t][i].steps);
        o.shi[t][i] = push(blob, h.sched_hinv[t][i].steps);
      }
      o.cs[i] = push(blob, h.crt_sum[i]);
      o.sb[i] = push(blob, h.sched_blind[i].steps);
    }
    o.el = push(blob, {(uint32_t)ks->e, (uint32_t)(ks->e >> 32)});
    o.dl = push(blob, h.d);
  }
  if (cudaMalloc(&ks->d_blob, blob.size() * 4) != cudaSuccess) return PMK_ENOMEM;
  if (cudaMemcpy(ks->d_blob, blob.data(), blob.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) return PMK_ECUDA;
  const uint32_t *b = ks->d_blob;
  // A schedule's device pointer, step count and highest table entry.
  auto view = [b](size_t off, const pmk::Schedule &sc, const uint32_t *&steps, uint32_t &nsteps, uint32_t &maxidx) {
    steps = b + off;
    nsteps = (uint32_t)sc.steps.size();
    maxidx = sc.maxidx;
  };
  std::vector<KeyDev> kd(ks->K);
  for (uint32_t k = 0; k < ks->K; k++) {
    const HostKey &h = ks->keys[k];
    const Offs &o = offs[k];
    KeyDev &d = kd[k];
    d = KeyDev{};
    d.N = b + o.N;
    d.R2 = b + o.R2;
    d.e_limbs = b + o.el;
    d.d_limbs = b + o.dl;
    d.n0 = h.n0;
    d.nprimes = h.nprimes;
    for (int t = 0; t < 2; t++) {
      view(o.se[t], h.sched_e[t], d.sched_e[t], d.nsteps_e[t], d.maxidx_e[t]);
      view(o.sd[t], h.sched_d[t], d.sched_d[t], d.nsteps_d[t], d.maxidx_d[t]);
    }
    for (uint32_t i = 0; i < h.nprimes; i++) {
      d.crt_sum[i] = b + o.cs[i];
      d.sched_blind[i] = b + o.sb[i];
      d.nsteps_blind[i] = (uint32_t)h.sched_blind[i].steps.size();
      d.maxa_blind[i] = h.sched_blind[i].maxa;
      d.maxb_blind[i] = h.sched_blind[i].maxb;
      d.P[i] = b + o.P[i];
      d.R2h[i] = b + o.R2h[i];
      d.R3h[i] = b + o.R3h[i];
      d.n0h[i] = h.n0h[i];
      for (int t = 0; t < 2; t++) {
        view(o.sh[t][i], h.sched_h[t][i], d.sched_h[t][i], d.nsteps_h[t][i], d.maxidx_h[t][i]);
        view(o.shi[t][i], h.sched_hinv[t][i], d.sched_hinv[t][i], d.nsteps_hinv[t][i], d.maxidx_hinv[t][i]);
      }
    }
  }
  if (cudaMalloc(&ks->d_keys, sizeof(KeyDev) * ks->K) != cudaSuccess) return PMK_ENOMEM;
  if (cudaMemcpy(ks->d_keys, kd.data(), sizeof(KeyDev) * ks->K, cudaMemcpyHostToDevice) != cudaSuccess)
    return PMK_ECUDA;
  return PMK_OK;
}

int finish_keyset(pmk_ctx *ctx, pmk_keyset *ks, pmk_keyset **out) {
  DeviceGuard g(ctx->device);
  int rc = g.ok() ? upload(ks) : PMK_ECUDA;
  if (rc != PMK_OK) {
    pmk_keyset_free(ks);
    return rc;
  }
  *out = ks;
  return PMK_OK;
}

bool width_built(uint32_t nbits, uint32_t nprimes = 2) {
  return pmk::default_config(nbits / 32, false).tpi != 0 && pmk::default_config(nbits / (32 * nprimes), true).tpi != 0;
}

// Most keys per key set: the CRT grid has one row per (key, prime) pair.
constexpr uint32_t kMaxKeys = 65535 / pmk::kMaxPrimes;

using pmk::kMaxChunks;

int check_chunk_call(const pmk_ctx *ctx, const pmk_keyset *ks, const void *in, const void *out, size_t n_chunks) {
  if (!ctx || !ks || n_chunks >= kMaxChunks) return PMK_EINVAL;
  if (ks->device != ctx->device) return PMK_EINVAL;
  if (!in || !out || !aligned16(in) || !aligned16(out)) return PMK_EINVAL;
  return PMK_OK;
}

// key_idx / groups / align: explicit key indices and their key-group table
// (launch_key_groups, with that alignment), or NULL for round robin (chunk
// t -> key t mod K).
int enqueue_encrypt(pmk_ctx *ctx, const pmk_keyset *ks, const uint32_t *in, uint32_t *out, size_t n, cudaStream_t st,
                    const uint32_t *key_idx = nullptr, const uint32_t *groups = nullptr,
                    uint32_t align = pmk::kGroupAlign) {
  const uint32_t S = ks->nbits / 32;
  int rc = pmk::launch_range_check(ks->d_keys, ks->K, S, in, n, ctx->d_status, st, key_idx);
  if (rc == PMK_OK)
    rc = pmk::launch_modexp(pmk::ExpMode::kEncrypt, S, cfg_for(ctx, S, false), ks->d_keys, ks->K, in, out, n, st,
                            ks->nprimes, groups, align);
  return rc;
}

// One residue per prime of each chunk (exponent d mod (r_i - 1), or r_i - 2
// for kCrtInverse) into out, then their recombination in place.
int enqueue_crt(pmk_ctx *ctx, const pmk_keyset *ks, pmk::ExpMode mode, const uint32_t *in, uint32_t *out, size_t n,
                cudaStream_t st, uint32_t *status_if_zero = nullptr, const uint32_t *groups = nullptr,
                uint32_t align = pmk::kGroupAlign) {
  const uint32_t b = ks->nprimes, H = ks->nbits / 32 / b;
  int rc = pmk::launch_modexp(mode, H, cfg_for(ctx, H, true), ks->d_keys, ks->K, in, out, n, st, b, groups, align);
  if (rc != PMK_OK) return rc;
  return pmk::launch_crt_sum(ks->nbits / 32, b, ks->d_keys, ks->K, out, n, st, status_if_zero, groups, align);
}

int enqueue_decrypt(pmk_ctx *ctx, const pmk_keyset *ks, const uint32_t *in, uint32_t *out, size_t n, int use_crt,
                    cudaStream_t st, const uint32_t *key_idx = nullptr, const uint32_t *groups = nullptr,
                    uint32_t align = pmk::kGroupAlign) {
  const uint32_t S = ks->nbits / 32;
  int rc = pmk::launch_range_check(ks->d_keys, ks->K, S, in, n, ctx->d_status, st, key_idx);
  if (rc != PMK_OK) return rc;
  if (!use_crt)
    return pmk::launch_modexp(pmk::ExpMode::kDecrypt, S, cfg_for(ctx, S, false), ks->d_keys, ks->K, in, out, n, st,
                              ks->nprimes, groups, align);
  return enqueue_crt(ctx, ks, pmk::ExpMode::kCrtHalf, in, out, n, st, nullptr, groups, align);
}

// The key-group alignment of a call: the largest instances-per-block of the
// kernels it launches, so that each key has at most one partly filled block
// per kernel (padding to more interleaves empty blocks with the working ones
// and can stack three working blocks on an SM where round robin puts two:
// 1.5x the time at 4096 bits and 1 MiB, measured).  0 when a width has no
// kernel.
uint32_t group_align(const pmk_ctx *ctx, const pmk_keyset *ks, bool use_crt) {
  const uint32_t S = ks->nbits / 32;
  if (!use_crt) return pmk::modexp_block_instances(S, cfg_for(ctx, S, false), false);
  const uint32_t H = S / ks->nprimes;
  return std::max(pmk::modexp_block_instances(H, cfg_for(ctx, H, true), true), pmk::crt_sum_block_instances(S));
}

// Explicit key indices: check them on the host side of the call, then build
// the key-group table in the context's staging on `st`.  *groups stays NULL
// for round robin.  Pair with release(ctx->grp, st) once the kernels reading
// the table are enqueued.
int key_groups_for(pmk_ctx *ctx, const pmk_keyset *ks, const uint32_t *key_idx, size_t n, cudaStream_t st,
                   uint32_t align, const uint32_t **groups) {
  *groups = nullptr;
  if (!key_idx) return PMK_OK;
  if (n >= pmk::kMaxGroupedChunks || (reinterpret_cast<uintptr_t>(key_idx) & 3u)) return PMK_EINVAL;
  if (align == 0) return PMK_EUNSUPPORTED;  // no kernel for this width
  int rc = acquire(ctx->grp, pmk::key_groups_words(n, ks->K) * 4, st);
  if (rc != PMK_OK) return rc;
  uint32_t *table = static_cast<uint32_t *>(ctx->grp.ptr);
  rc = pmk::launch_key_groups(key_idx, n, ks->K, align, table, ctx->d_status, st);
  if (rc == PMK_OK) *groups = table;
  return rc;
}

}  // namespace

namespace pmk {
bool fault_injected(const char *site) {
  const char *v = std::getenv("PMK_INJECT_FAULT");
  return v && std::strcmp(v, site) == 0;
}
}  // namespace pmk

extern "C" {

int pmk_create(pmk_ctx **out, int cuda_device) {
  if (!out) return PMK_EINVAL;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess) return PMK_ECUDA;
  if (cuda_device < 0 || cuda_device >= count) return PMK_EINVAL;
  pmk_ctx *ctx = new (std::nothrow) pmk_ctx();
  if (!ctx) return PMK_ENOMEM;
  ctx->device = cuda_device;
  DeviceGuard g(cuda_device);
  if (!g.ok()) {
    delete ctx;
    return PMK_ECUDA;
  }
  if (cudaMalloc(&ctx->d_status, pmk::kStatusRecordBytes) != cudaSuccess ||
      pmk::clear_status(ctx->d_status, nullptr) != PMK_OK || cudaStreamSynchronize(nullptr) != cudaSuccess) {
    pmk_destroy(ctx);
    return PMK_ENOMEM;
  }
  *out = ctx;
  return PMK_OK;
}

void pmk_destroy(pmk_ctx *ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  drop(ctx->msg);
  drop(ctx->a);
  drop(ctx->b);
  drop(ctx->grp);
  cudaFree(ctx->d_status);
  delete ctx;
}

int pmk_keygen(pmk_ctx *ctx, uint32_t K, uint32_t nbits, uint64_t e, uint64_t seed, pmk_keyset **out) {
  return pmk_keygen_multiprime(ctx, K, nbits, 2, e, seed, out);
}

int pmk_keygen_multiprime(pmk_ctx *ctx, uint32_t K, uint32_t nbits, uint32_t nprimes, uint64_t e, uint64_t seed,
                          pmk_keyset **out) {
  pmk::TraceRange trace("pmk_keygen_multiprime");
  if (!ctx || !out) return PMK_EINVAL;
  if (K == 0 || K > kMaxKeys || !pmk::valid_multiprime(nbits, nprimes) || e < 3 || !(e & 1) || (e >> 32))
    return PMK_EINVAL;
  if (!width_built(nbits, nprimes)) return PMK_EUNSUPPORTED;
  try {
    pmk_keyset *ks = new pmk_keyset();
    ks->device = ctx->device;
    ks->K = K;
    ks->nbits = nbits;
    ks->e = e;
    ks->nprimes = nprimes;
    int rc = pmk::host_keygen_mp(K, nbits, nprimes, e, seed, ks->keys);
    if (rc != PMK_OK) {
      delete ks;
      return rc;
    }
    return finish_keyset(ctx, ks, out);
  } catch (const std::bad_alloc &) {
    return PMK_ENOMEM;
  }
}

int pmk_keygen_host_multiprime(uint32_t K, uint32_t nbits, uint32_t nprimes, uint64_t e, uint64_t seed, uint32_t *N,
                               uint32_t *d, uint32_t *primes, uint32_t *dexp, uint32_t *coef) {
  if (K == 0 || K > kMaxKeys || !pmk::valid_multiprime(nbits, nprimes) || e < 3 || !(e & 1) || (e >> 32))
    return PMK_EINVAL;
  try {
    pmk_keyset ks;
    ks.K = K;
    ks.nbits = nbits;
    ks.e = e;
    ks.nprimes = nprimes;
    int rc = pmk::host_keygen_mp(K, nbits, nprimes, e, seed, ks.keys);
    if (rc == PMK_OK) rc = pmk_keyset_export_fields(&ks, N, d, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (rc == PMK_OK) rc = pmk_keyset_export_primes(&ks, primes, dexp, coef);
    return rc;
  } catch (const std::bad_alloc &) {
    return PMK_ENOMEM;
  }
}

int pmk_keygen_host(uint32_t K, uint32_t nbits, uint64_t e, uint64_t seed, uint32_t *N, uint32_t *d, uint32_t *p,
                    uint32_t *q, uint32_t *dp, uint32_t *dq, uint32_t *qinv) {
  if (K == 0 || K > kMaxKeys || nbits < 128 || nbits > 8192 || nbits % 128 || e < 3 || !(e & 1) || (e >> 32))
    return PMK_EINVAL;
  try {
    pmk_keyset ks;
    ks.K = K;
    ks.nbits = nbits;
    ks.e = e;
    int rc = pmk::host_keygen(K, nbits, e, seed, ks.keys);
    if (rc != PMK_OK) return rc;
    return pmk_keyset_export_fields(&ks, N, d, p, q, dp, dq, qinv);
  } catch (const std::bad_alloc &) {
    return PMK_ENOMEM;
  }
}

int pmk_keyset_from_primes(pmk_ctx *ctx, uint32_t K, uint32_t nbits, uint64_t e, const uint32_t *p,
                           const uint32_t *q, pmk_keyset **out) {
  pmk::TraceRange trace("pmk_keyset_from_primes");
  if (!ctx || !out || !p || !q || K == 0 || K > kMaxKeys) return PMK_EINVAL;
  if (nbits < 128 || nbits > 8192 || nbits % 128 || e < 3 || !(e & 1) || (e >> 32)) return PMK_EINVAL;
  if (!width_built(nbits)) return PMK_EUNSUPPORTED;
  try {
    pmk_keyset *ks = new pmk_keyset();
    ks->device = ctx->device;
    ks->K = K;
    ks->nbits = nbits;
    ks->e = e;
    ks->keys.resize(K);
    const size_t h = nbits / 64;
    for (uint32_t k = 0; k < K; k++) {
      int rc = pmk::host_from_primes(nbits, e, p + k * h, q + k * h, ks->keys[k]);
      if (rc != PMK_OK) {
        delete ks;
        return rc;
      }
    }
    return finish_keyset(ctx, ks, out);
  } catch (const std::bad_alloc &) {
    return PMK_ENOMEM;
  }
}

int pmk_keyset_from_primes_multi(pmk_ctx *ctx, uint32_t K, uint32_t nbits, uint32_t nprimes, uint64_t e,
                                 const uint32_t *primes, pmk_keyset **out) {
  pmk::TraceRange trace("pmk_keyset_from_primes_multi");
  if (!ctx || !out || !primes || K == 0 || K > kMaxKeys) return PMK_EINVAL;
  if (!pmk::valid_multiprime(nbits, nprimes) || e < 3 || !(e & 1) || (e >> 32)) return PMK_EINVAL;
  if (!width_built(nbits, nprimes)) return PMK_EUNSUPPORTED;
  try {
    pmk_keyset *ks = new pmk_keyset();
    ks->device = ctx->device;
    ks->K = K;
    ks->nbits = nbits;
    ks->e = e;
    ks->nprimes = nprimes;
    ks->keys.resize(K);
    const size_t s = nbits / 32;
    for (uint32_t k = 0; k < K; k++) {
      int rc = pmk::host_from_primes_mp(nbits, nprimes, e, primes + k * s, ks->keys[k]);
      if (rc != PMK_OK) {
        delete ks;
        return rc;
      }
    }
    return finish_keyset(ctx, ks, out);
  } catch (const std::bad_alloc &) {
    return PMK_ENOMEM;
  }
}

int pmk_keyset_export_fields(const pmk_keyset *ks, uint32_t *N, uint32_t *d, uint32_t *p, uint32_t *q, uint32_t *dp,
                      uint32_t *dq, uint32_t *qinv) {
  if (!ks) return PMK_EINVAL;
  if (ks->nprimes != 2 && (p || q || dp || dq || qinv)) return PMK_EINVAL;  // primes: pmk_keyset_export_primes
  const size_t s = ks->nbits / 32, h = s / 2;
  for (uint32_t k = 0; k < ks->K; k++) {
    const HostKey &x = ks->keys[k];
    if (N) std::memcpy(N + k * s, x.N.data(), s * 4);
    if (d) std::memcpy(d + k * s, x.d.data(), s * 4);
    if (p) std::memcpy(p + k * h, x.p.data(), h * 4);
    if (q) std::memcpy(q + k * h, x.q.data(), h * 4);
    if (dp) std::memcpy(dp + k * h, x.dp.data(), h * 4);
    if (dq) std::memcpy(dq + k * h, x.dq.data(), h * 4);
    if (qinv) std::memcpy(qinv + k * h, x.qinv.data(), h * 4);
  }
  return PMK_OK;
}

int pmk_keyset_export_primes(const pmk_keyset *ks, uint32_t *primes, uint32_t *dexp, uint32_t *coef) {
  if (!ks) return PMK_EINVAL;
  const size_t s = ks->nbits / 32, b = ks->nprimes, h = s / b;
  for (uint32_t k = 0; k < ks->K; k++) {
    const HostKey &x = ks->keys[k];
    for (size_t i = 0; i < b; i++) {
      if (primes) std::memcpy(primes + k * s + i * h, x.pr[i].data(), h * 4);
      if (dexp) std::memcpy(dexp + k * s + i * h, x.dpr[i].data(), h * 4);
      if (coef) {
        if (i == 1) std::memset(coef + k * s + i * h, 0, h * 4);
        else std::memcpy(coef + k * s + i * h, x.coef[i].data(), h * 4);
      }
    }
  }
  return PMK_OK;
}

// ---- key-set blob: a versioned, little-endian serialisation (pmkrsa.h).
}  // extern "C"

namespace {

constexpr uint32_t kBlobVersion = 1;
constexpr size_t kBlobHeader = 32, kBlobTrailer = 8;
constexpr uint32_t kBlobFields = 5;  // N, d, primes, dexp, coef: nbits/32 limbs each

size_t blob_size(uint32_t K, uint32_t nbits) {
  return kBlobHeader + (size_t)K * kBlobFields * (nbits / 32) * 4 + kBlobTrailer;
}

void put32(unsigned char *p, uint32_t v) {
  for (int i = 0; i < 4; i++) p[i] = (unsigned char)(v >> (8 * i));
}
void put64(unsigned char *p, uint64_t v) {
  for (int i = 0; i < 8; i++) p[i] = (unsigned char)(v >> (8 * i));
}
uint32_t get32(const unsigned char *p) {
  uint32_t v = 0;
  for (int i = 3; i >= 0; i--) v = (v << 8) | p[i];
  return v;
}
uint64_t get64(const unsigned char *p) {
  uint64_t v = 0;
  for (int i = 7; i >= 0; i--) v = (v << 8) | p[i];
  return v;
}

// FNV-1a, 64-bit (the published offset basis and prime), over a byte range.
uint64_t fnv1a64(const unsigned char *p, size_t n) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (size_t i = 0; i < n; i++) {
    h ^= p[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

// The five per-key fields in blob order, as s-limb rows (primes, dexp, coef
// hold b values of s/b limbs each, the layout of pmk_keyset_export_primes).
void key_rows(const pmk::HostKey &x, uint32_t nbits, uint32_t b, std::vector<uint32_t> &rows) {
  const size_t s = nbits / 32, h = s / b;
  rows.assign(kBlobFields * s, 0u);
  std::copy(x.N.begin(), x.N.end(), rows.begin());
  std::copy(x.d.begin(), x.d.end(), rows.begin() + s);
  for (size_t i = 0; i < b; i++) {
    std::copy(x.pr[i].begin(), x.pr[i].end(), rows.begin() + 2 * s + i * h);
    std::copy(x.dpr[i].begin(), x.dpr[i].end(), rows.begin() + 3 * s + i * h);
    if (i != 1) std::copy(x.coef[i].begin(), x.coef[i].end(), rows.begin() + 4 * s + i * h);
  }
}

}  // namespace

extern "C" {

int pmk_keyset_export(const pmk_keyset *ks, void *buf, size_t *len) {
  if (!ks || !len) return PMK_EINVAL;
  const size_t need = blob_size(ks->K, ks->nbits);
  if (!buf) {
    *len = need;
    return PMK_OK;
  }
  if (*len < need) {
    *len = need;
    return PMK_EINVAL;
  }
  unsigned char *p = static_cast<unsigned char *>(buf);
  std::memcpy(p, "PMKK", 4);
  put32(p + 4, kBlobVersion);
  put32(p + 8, ks->K);
  put32(p + 12, ks->nbits);
  put32(p + 16, ks->nprimes);
  put32(p + 20, 0);
  put64(p + 24, ks->e);
  size_t off = kBlobHeader;
  std::vector<uint32_t> rows;
  for (uint32_t k = 0; k < ks->K; k++) {
    key_rows(ks->keys[k], ks->nbits, ks->nprimes, rows);
    for (uint32_t w : rows) {
      put32(p + off, w);
      off += 4;
    }
  }
  put64(p + off, fnv1a64(p, off));
  *len = need;
  return PMK_OK;
}

int pmk_keyset_import(pmk_ctx *ctx, const void *buf, size_t len, pmk_keyset **out) {
  pmk::TraceRange trace("pmk_keyset_import");
  if (!buf || !out || len < kBlobHeader + kBlobTrailer) return PMK_EINVAL;
  const unsigned char *p = static_cast<const unsigned char *>(buf);
  if (std::memcmp(p, "PMKK", 4) != 0 || get32(p + 4) != kBlobVersion || get32(p + 20) != 0) return PMK_EINVAL;
  const uint32_t K = get32(p + 8), nbits = get32(p + 12), b = get32(p + 16);
  const uint64_t e = get64(p + 24);
  if (K == 0 || K > kMaxKeys || !pmk::valid_multiprime(nbits, b) || e < 3 || !(e & 1) || (e >> 32)) return PMK_EINVAL;
  if (len != blob_size(K, nbits) || get64(p + len - kBlobTrailer) != fnv1a64(p, len - kBlobTrailer))
    return PMK_EINVAL;
  if (ctx && !width_built(nbits, b)) return PMK_EUNSUPPORTED;
  try {
    pmk_keyset *ks = new pmk_keyset();
    ks->device = ctx ? ctx->device : -1;
    ks->K = K;
    ks->nbits = nbits;
    ks->e = e;
    ks->nprimes = b;
    ks->keys.resize(K);
    const size_t s = nbits / 32;
    std::vector<uint32_t> stored(kBlobFields * s), derived;
    for (uint32_t k = 0; k < K; k++) {
      const unsigned char *q = p + kBlobHeader + (size_t)k * kBlobFields * s * 4;
      for (size_t i = 0; i < stored.size(); i++) stored[i] = get32(q + 4 * i);
      // Everything is derived again from the primes; the stored N, d and CRT
      // values must agree with it, or the blob is refused.
      int rc = pmk::host_from_primes_mp(nbits, b, e, stored.data() + 2 * s, ks->keys[k]);
      if (rc == PMK_OK) {
        key_rows(ks->keys[k], nbits, b, derived);
        if (derived != stored) rc = PMK_EINVAL;
      }
      if (rc != PMK_OK) {
        delete ks;
        return rc;
      }
    }
    if (!ctx) {  // host only: exportable, not usable by device calls
      *out = ks;
      return PMK_OK;
    }
    return finish_keyset(ctx, ks, out);
  } catch (const std::bad_alloc &) {
    return PMK_ENOMEM;
  }
}

uint32_t pmk_keyset_num_primes(const pmk_keyset *ks) { return ks ? ks->nprimes : 0; }
uint32_t pmk_keyset_num_keys(const pmk_keyset *ks) { return ks ? ks->K : 0; }
uint32_t pmk_keyset_nbits(const pmk_keyset *ks) { return ks ? ks->nbits : 0; }
uint64_t pmk_keyset_e(const pmk_keyset *ks) { return ks ? ks->e : 0; }

void pmk_keyset_free(pmk_keyset *ks) {
  if (!ks) return;
  if (ks->device >= 0) {
    DeviceGuard g(ks->device);
    cudaFree(ks->d_blob);
    cudaFree(ks->d_keys);
  }
  delete ks;
}

size_t pmk_payload_bytes(uint32_t nbits) { return nbits >= 16 ? nbits / 8 - 1 : 0; }

size_t pmk_num_chunks(size_t msg_len, uint32_t nbits) {
  const size_t P = pmk_payload_bytes(nbits);
  return P ? (msg_len + P - 1) / P : 0;
}

int pmk_split(pmk_ctx *ctx, uint32_t nbits, const uint8_t *d_msg, size_t msg_len, uint32_t *d_chunks, size_t n_chunks,
              void *stream) {
  pmk::TraceRange trace("pmk_split");
  if (!ctx || nbits < 128 || nbits % 128 || nbits > 8192) return PMK_EINVAL;
  if (n_chunks != pmk_num_chunks(msg_len, nbits) || n_chunks >= kMaxChunks) return PMK_EINVAL;
  if (n_chunks == 0) return PMK_OK;
  if (!d_msg || !d_chunks) return PMK_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok()) return PMK_ECUDA;
  return pmk::launch_split(nbits, d_msg, msg_len, d_chunks, n_chunks, as_stream(stream));
}

int pmk_join(pmk_ctx *ctx, uint32_t nbits, const uint32_t *d_chunks, size_t n_chunks, uint8_t *d_msg, size_t msg_len,
             void *stream) {
  pmk::TraceRange trace("pmk_join");
  if (!ctx || nbits < 128 || nbits % 128 || nbits > 8192) return PMK_EINVAL;
  if (n_chunks != pmk_num_chunks(msg_len, nbits) || n_chunks >= kMaxChunks) return PMK_EINVAL;
  if (msg_len == 0) return PMK_OK;
  if (!d_msg || !d_chunks) return PMK_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok()) return PMK_ECUDA;
  return pmk::launch_join(nbits, d_chunks, n_chunks, d_msg, msg_len, as_stream(stream));
}

int pmk_encrypt_chunks(pmk_ctx *ctx, const pmk_keyset *ks, const uint32_t *d_in, uint32_t *d_out, size_t n_chunks,
                       const uint32_t *d_key_idx, void *stream) {
  pmk::TraceRange trace("pmk_encrypt_chunks");
  if (n_chunks == 0) return (ctx && ks && ks->device == ctx->device) ? PMK_OK : PMK_EINVAL;
  int rc = check_chunk_call(ctx, ks, d_in, d_out, n_chunks);
  if (rc != PMK_OK) return rc;
  DeviceGuard g(ctx->device);
  if (!g.ok()) return PMK_ECUDA;
  cudaStream_t st = as_stream(stream);
  const uint32_t *groups = nullptr;
  const uint32_t align = d_key_idx ? group_align(ctx, ks, false) : pmk::kGroupAlign;
  rc = key_groups_for(ctx, ks, d_key_idx, n_chunks, st, align, &groups);
  if (rc == PMK_OK) rc = enqueue_encrypt(ctx, ks, d_in, d_out, n_chunks, st, d_key_idx, groups, align);
  if (d_key_idx) release(ctx->grp, st);
  return rc;
}

int pmk_decrypt_chunks(pmk_ctx *ctx, const pmk_keyset *ks, const uint32_t *d_in, uint32_t *d_out, size_t n_chunks,
                       const uint32_t *d_key_idx, int use_crt, void *stream) {
  pmk::TraceRange trace("pmk_decrypt_chunks");
  if (n_chunks == 0) return (ctx && ks && ks->device == ctx->device) ? PMK_OK : PMK_EINVAL;
  int rc = check_chunk_call(ctx, ks, d_in, d_out, n_chunks);
  if (rc != PMK_OK) return rc;
  const size_t bytes = n_chunks * (ks->nbits / 8);
  if (use_crt && overlap(d_in, bytes, d_out, bytes)) return PMK_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok()) return PMK_ECUDA;
  cudaStream_t st = as_stream(stream);
  const uint32_t *groups = nullptr;
  const uint32_t align = d_key_idx ? group_align(ctx, ks, use_crt != 0) : pmk::kGroupAlign;
  rc = key_groups_for(ctx, ks, d_key_idx, n_chunks, st, align, &groups);
  if (rc == PMK_OK) rc = enqueue_decrypt(ctx, ks, d_in, d_out, n_chunks, use_crt, st, d_key_idx, groups, align);
  if (d_key_idx) release(ctx->grp, st);
  return rc;
}

int pmk_encrypt_blinded(pmk_ctx *ctx, const pmk_keyset *ks, const uint32_t *d_m, const uint32_t *d_r,
                        uint32_t *d_cstar, uint32_t *d_cr, size_t n_chunks, void *stream) {
  pmk::TraceRange trace("pmk_encrypt_blinded");
  if (n_chunks == 0) return (ctx && ks && ks->device == ctx->device) ? PMK_OK : PMK_EINVAL;
  int rc = check_chunk_call(ctx, ks, d_m, d_cstar, n_chunks);
  if (rc == PMK_OK) rc = check_chunk_call(ctx, ks, d_r, d_cr, n_chunks);
  if (rc != PMK_OK) return rc;
  const size_t bytes = n_chunks * (ks->nbits / 8);
  const void *bufs[4] = {d_m, d_r, d_cstar, d_cr};
  for (int i = 0; i < 4; i++)
    for (int j = i + 1; j < 4; j++)
      if (overlap(bufs[i], bytes, bufs[j], bytes)) return PMK_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok()) return PMK_ECUDA;
  cudaStream_t st = as_stream(stream);
  const uint32_t S = ks->nbits / 32;
  rc = enqueue_encrypt(ctx, ks, d_m, d_cstar, n_chunks, st);                     // c = m^e (into C*)
  if (rc == PMK_OK) rc = enqueue_encrypt(ctx, ks, d_r, d_cr, n_chunks, st);     // c_r = r^e
  if (rc == PMK_OK) rc = pmk::launch_mulmod(S, ks->d_keys, ks->K, d_cstar, d_cr, d_cstar, n_chunks, st);  // c* = c c_r
  return rc;
}

int pmk_decrypt_blinded(pmk_ctx *ctx, const pmk_keyset *ks, const uint32_t *d_cstar, const uint32_t *d_cr,
                        uint32_t *d_m, size_t n_chunks, int use_crt, void *stream) {
  pmk::TraceRange trace("pmk_decrypt_blinded");
  if (n_chunks == 0) return (ctx && ks && ks->device == ctx->device) ? PMK_OK : PMK_EINVAL;
  int rc = check_chunk_call(ctx, ks, d_cstar, d_m, n_chunks);
  if (rc == PMK_OK) rc = check_chunk_call(ctx, ks, d_cr, d_m, n_chunks);
  if (rc != PMK_OK) return rc;
  const size_t bytes = n_chunks * (ks->nbits / 8);
  if (overlap(d_cstar, bytes, d_m, bytes) || overlap(d_cr, bytes, d_m, bytes) || overlap(d_cstar, bytes, d_cr, bytes))
    return PMK_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok()) return PMK_ECUDA;
  cudaStream_t st = as_stream(stream);
  const uint32_t S = ks->nbits / 32, H = S / ks->nprimes;
  rc = pmk::launch_range_check(ks->d_keys, ks->K, S, d_cstar, n_chunks, ctx->d_status, st);
  if (rc == PMK_OK) rc = pmk::launch_range_check(ks->d_keys, ks->K, S, d_cr, n_chunks, ctx->d_status, st);
  if (rc != PMK_OK) return rc;
  if (use_crt && pmk::blind_crt_built(H)) {
    // per prime: c*^(d_i) c_r^(r_i - 1 - d_i) = (c* c_r^-1)^d mod r_i in one
    // joint exponentiation, then the recombination
    rc = pmk::launch_blind_crt(H, ks->nprimes, ks->d_keys, ks->K, d_cstar, d_cr, d_m, n_chunks, st, ctx->d_status);
    if (rc == PMK_OK) rc = pmk::launch_crt_sum(S, ks->nprimes, ks->d_keys, ks->K, d_m, n_chunks, st);
    return rc;
  }
  // c_r^-1 mod N: Fermat inverses mod each prime, recombined (into d_m)
  rc = enqueue_crt(ctx, ks, pmk::ExpMode::kCrtInverse, d_cr, d_m, n_chunks, st, ctx->d_status);
  // x = c* c_r^-1, in place
  if (rc == PMK_OK) rc = pmk::launch_mulmod(S, ks->d_keys, ks->K, d_cstar, d_m, d_m, n_chunks, st);
  if (rc != PMK_OK) return rc;
  // m = x^d
  if (!use_crt)
    return pmk::launch_modexp(pmk::ExpMode::kDecrypt, S, cfg_for(ctx, S, false), ks->d_keys, ks->K, d_m, d_m,
                              n_chunks, st);
  rc = acquire(ctx->b, n_chunks * S * 4, st);
  uint32_t *x = static_cast<uint32_t *>(ctx->b.ptr);
  if (rc == PMK_OK && cudaMemcpyAsync(x, d_m, n_chunks * S * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    rc = PMK_ECUDA;
  if (rc == PMK_OK) rc = enqueue_crt(ctx, ks, pmk::ExpMode::kCrtHalf, x, d_m, n_chunks, st);
  release(ctx->b, st);
  return rc;
}

int pmk_modexp_chunks_baseline(pmk_ctx *ctx, const pmk_keyset *ks, const uint32_t *d_in, uint32_t *d_out,
                               size_t n_chunks, int decrypt, void *stream) {
  pmk::TraceRange trace("pmk_modexp_chunks_baseline");
  if (n_chunks == 0) return (ctx && ks && ks->device == ctx->device) ? PMK_OK : PMK_EINVAL;
  int rc = check_chunk_call(ctx, ks, d_in, d_out, n_chunks);
  if (rc != PMK_OK) return rc;
  DeviceGuard g(ctx->device);
  if (!g.ok()) return PMK_ECUDA;
  const uint32_t S = ks->nbits / 32;
  rc = pmk::launch_range_check(ks->d_keys, ks->K, S, d_in, n_chunks, ctx->d_status, as_stream(stream));
  if (rc == PMK_OK)
    rc = pmk::launch_modexp_naive(!decrypt, S, ks->d_keys, ks->K, d_in, d_out, n_chunks, as_stream(stream));
  return rc;
}

int pmk_sync_status_detail(pmk_ctx *ctx, void *stream, uint64_t *first_chunk) {
  pmk::TraceRange trace("pmk_sync_status_detail");
  if (first_chunk) *first_chunk = UINT64_MAX;
  if (!ctx) return PMK_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok()) return PMK_ECUDA;
  if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return PMK_ECUDA;
  uint32_t rec[4] = {0, 0, 0, 0};
  if (cudaMemcpy(rec, ctx->d_status, sizeof rec, cudaMemcpyDeviceToHost) != cudaSuccess) return PMK_ECUDA;
  const uint32_t st = rec[0];
  if (st == 0) return PMK_OK;
  if (first_chunk) *first_chunk = (uint64_t)rec[2] | ((uint64_t)rec[3] << 32);
  if (pmk::clear_status(ctx->d_status, nullptr) != PMK_OK || cudaStreamSynchronize(nullptr) != cudaSuccess)
    return PMK_ECUDA;
  if (st & pmk::kStatusKeyIndex) return PMK_EKEYINDEX;
  if (st & pmk::kStatusRange) return PMK_ERANGE;
  return (st & pmk::kStatusNotInvertible) ? PMK_ENOINV : PMK_ECUDA;
}

int pmk_sync_status(pmk_ctx *ctx, void *stream) { return pmk_sync_status_detail(ctx, stream, nullptr); }

int pmk_encrypt_message_host(pmk_ctx *ctx, const pmk_keyset *ks, const uint8_t *h_msg, size_t msg_len,
                             uint32_t *h_cipher, size_t n_chunks, void *stream) {
  pmk::TraceRange trace("pmk_encrypt_message_host");
  if (!ctx || !ks || ks->device != ctx->device) return PMK_EINVAL;
  if (n_chunks != pmk_num_chunks(msg_len, ks->nbits) || n_chunks >= kMaxChunks) return PMK_EINVAL;
  if (n_chunks == 0) return PMK_OK;
  if (!h_msg || !h_cipher) return PMK_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok()) return PMK_ECUDA;
  const size_t words = n_chunks * (ks->nbits / 32);
  cudaStream_t st = as_stream(stream);
  int rc = acquire(ctx->msg, msg_len, st);
  if (rc == PMK_OK) rc = acquire(ctx->a, words * 4, st);
  uint8_t *m = static_cast<uint8_t *>(ctx->msg.ptr);
  uint32_t *c = static_cast<uint32_t *>(ctx->a.ptr);
  bool queued = false;  // a copy from or to the caller's host memory is in flight
  if (rc == PMK_OK) {
    queued = true;
    if (cudaMemcpyAsync(m, h_msg, msg_len, cudaMemcpyHostToDevice, st) != cudaSuccess) rc = PMK_ECUDA;
  }
  if (rc == PMK_OK && pmk::fault_injected("after_copy")) rc = PMK_ECUDA;
  if (rc == PMK_OK) rc = pmk::launch_split(ks->nbits, m, msg_len, c, n_chunks, st);
  if (rc == PMK_OK) rc = enqueue_encrypt(ctx, ks, c, c, n_chunks, st);
  if (rc == PMK_OK && cudaMemcpyAsync(h_cipher, c, words * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    rc = PMK_ECUDA;
  release(ctx->msg, st);
  release(ctx->a, st);
  if (rc != PMK_OK) {
    if (queued) cudaStreamSynchronize(st);  // return with no copy of the caller's buffers in flight
    return rc;
  }
  return pmk_sync_status(ctx, stream);
}

int pmk_decrypt_message_host(pmk_ctx *ctx, const pmk_keyset *ks, const uint32_t *h_cipher, size_t n_chunks,
                             uint8_t *h_msg, size_t msg_len, int use_crt, void *stream) {
  pmk::TraceRange trace("pmk_decrypt_message_host");
  if (!ctx || !ks || ks->device != ctx->device) return PMK_EINVAL;
  if (n_chunks != pmk_num_chunks(msg_len, ks->nbits) || n_chunks >= kMaxChunks) return PMK_EINVAL;
  if (n_chunks == 0) return PMK_OK;
  if (!h_msg || !h_cipher) return PMK_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok()) return PMK_ECUDA;
  const size_t words = n_chunks * (ks->nbits / 32);
  cudaStream_t st = as_stream(stream);
  int rc = acquire(ctx->msg, msg_len, st);
  if (rc == PMK_OK) rc = acquire(ctx->a, words * 4, st);
  if (rc == PMK_OK) rc = acquire(ctx->b, words * 4, st);
  uint8_t *m = static_cast<uint8_t *>(ctx->msg.ptr);
  uint32_t *c = static_cast<uint32_t *>(ctx->a.ptr), *p = static_cast<uint32_t *>(ctx->b.ptr);
  bool queued = false;  // a copy from or to the caller's host memory is in flight
  if (rc == PMK_OK) {
    queued = true;
    if (cudaMemcpyAsync(c, h_cipher, words * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) rc = PMK_ECUDA;
  }
  if (rc == PMK_OK && pmk::fault_injected("after_copy")) rc = PMK_ECUDA;
  if (rc == PMK_OK) rc = enqueue_decrypt(ctx, ks, c, p, n_chunks, use_crt, st);
  if (rc == PMK_OK) rc = pmk::launch_join(ks->nbits, p, n_chunks, m, msg_len, st);
  if (rc == PMK_OK && cudaMemcpyAsync(h_msg, m, msg_len, cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = PMK_ECUDA;
  release(ctx->msg, st);
  release(ctx->a, st);
  release(ctx->b, st);
  if (rc != PMK_OK) {
    if (queued) cudaStreamSynchronize(st);  // return with no copy of the caller's buffers in flight
    return rc;
  }
  return pmk_sync_status(ctx, stream);
}

const char *pmk_strerror(int code) {
  switch (code) {
    case PMK_OK: return "ok";
    case PMK_EINVAL: return "invalid argument";
    case PMK_ERANGE: return "input chunk not below its modulus";
    case PMK_ENOMEM: return "out of memory";
    case PMK_ECUDA: return "CUDA runtime error";
    case PMK_EUNSUPPORTED: return "key width or launch geometry not built";
    case PMK_ETOOLARGE: return "request exceeds the fixed capacity of the allocation-free call";
    case PMK_ENOINV: return "blinding value not invertible modulo its key";
    case PMK_EKEYINDEX: return "key index not below the key set's key count";
    default: return "unknown error";
  }
}

int pmk_measure_int_peak(pmk_ctx *ctx, double *macs_per_clk_per_sm, double *sm_mhz, int *num_sms) {
  if (!ctx || !macs_per_clk_per_sm || !sm_mhz || !num_sms) return PMK_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok()) return PMK_ECUDA;
  return pmk::measure_int_peak(macs_per_clk_per_sm, sm_mhz, num_sms);
}

int pmk_measure_imad_peak(pmk_ctx *ctx, double *mad_lo_per_clk_per_sm, double *sm_mhz, int *num_sms) {
  if (!ctx || !mad_lo_per_clk_per_sm || !sm_mhz || !num_sms) return PMK_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok()) return PMK_ECUDA;
  return pmk::measure_imad_peak(mad_lo_per_clk_per_sm, sm_mhz, num_sms);
}

int pmk_set_kernel_config(pmk_ctx *ctx, uint32_t limbs, int crt, uint32_t tpi, uint32_t form) {
  if (!ctx) return PMK_EINVAL;
  const uint32_t key = limbs << 1 | (crt ? 1u : 0u);
  if (tpi == 0) {
    ctx->cfg.erase(key);
    return PMK_OK;
  }
  const pmk::KernelConfig c{tpi, form};
  if (!pmk::modexp_built(limbs, c, crt != 0)) return PMK_EUNSUPPORTED;
  ctx->cfg[key] = c;
  return PMK_OK;
}

int pmk_get_kernel_config(const pmk_ctx *ctx, uint32_t limbs, int crt, uint32_t *tpi, uint32_t *form) {
  if (!ctx || !tpi || !form) return PMK_EINVAL;
  const pmk::KernelConfig c = cfg_for(ctx, limbs, crt != 0);
  if (c.tpi == 0) return PMK_EUNSUPPORTED;
  *tpi = c.tpi;
  *form = c.form;
  return PMK_OK;
}

int pmk_set_kernel_window(pmk_ctx *ctx, uint32_t limbs, int crt, uint32_t max_window) {
  if (!ctx || (max_window != 0 && max_window != pmk::kWindowFull && max_window != pmk::kWindowSmall))
    return PMK_EINVAL;
  if (pmk::list_configs(limbs, crt != 0, nullptr, 0) <= 0) return PMK_EUNSUPPORTED;
  if (max_window == pmk::kWindowSmall && !small_table_available(limbs, crt != 0)) return PMK_EUNSUPPORTED;
  const uint32_t key = limbs << 1 | (crt ? 1u : 0u);
  if (max_window == pmk::kWindowSmall)
    ctx->table[key] = pmk::kTableSmall;
  else
    ctx->table.erase(key);
  return PMK_OK;
}

int pmk_get_kernel_window(const pmk_ctx *ctx, uint32_t limbs, int crt, uint32_t *max_window) {
  if (!ctx || !max_window) return PMK_EINVAL;
  if (pmk::list_configs(limbs, crt != 0, nullptr, 0) <= 0) return PMK_EUNSUPPORTED;
  *max_window = pmk::window_of(cfg_for(ctx, limbs, crt != 0).table);
  return PMK_OK;
}

int pmk_list_kernel_configs(uint32_t limbs, int crt, uint32_t *tpi, uint32_t *form, int max) {
  if (max < 0) return PMK_EINVAL;
  std::vector<pmk::KernelConfig> v(max > 0 ? max : 1);
  const int n = pmk::list_configs(limbs, crt != 0, v.data(), max);
  for (int i = 0; i < n && i < max; i++) {
    if (tpi) tpi[i] = v[i].tpi;
    if (form) form[i] = v[i].form;
  }
  return n;
}

}  // extern "C"
