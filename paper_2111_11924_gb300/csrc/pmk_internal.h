// Internal declarations shared by the host code and the CUDA kernels of the
// PMKRSA library.  Nothing here is part of the C ABI (include/pmkrsa.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "pmkrsa.h"

namespace pmk {

// An NVTX range named after a C ABI entry point, open for the call's host
// duration: profilers (ncu --nvtx, nsys) attribute the call's launches to it.
// Without a profiler attached the push / pop are no-ops.
class TraceRange {
 public:
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

// Error bits written by kernels into word 0 of the context's device status record.
enum : uint32_t { kStatusRange = 1u, kStatusNotInvertible = 2u, kStatusKeyIndex = 4u };

// The device status record of a context (16 bytes, 8-byte aligned): word 0
// holds the error bits, words 2-3 the smallest chunk index (within its call)
// that raised one, all ones when none.  Kernels receive a pointer to word 0.
constexpr size_t kStatusRecordBytes = 16;
constexpr unsigned long long kNoErrorChunk = ~0ull;
#ifdef __CUDACC__
// Record error `flag` for chunk t.
__device__ __forceinline__ void report(uint32_t *status, uint32_t flag, long long t) {
  atomicOr(status, flag);
  atomicMin(reinterpret_cast<unsigned long long *>(status + 2), (unsigned long long)t);
}
#endif
// Clear a status record on `st` (error bits 0, no failing chunk).
int clear_status(uint32_t *status, cudaStream_t st);

// Key groups (explicit key indices): each key's chunks occupy a segment of
// slots padded to a multiple of the table's alignment (a power of two, at
// most kGroupAlign); a padding slot holds kNoChunk.
constexpr uint32_t kGroupAlign = 64;
constexpr uint32_t kNoChunk = 0xffffffffu;
// Most chunks of a call with explicit key indices (slot numbers stay 32-bit).
constexpr size_t kMaxGroupedChunks = (size_t)1 << 31;

// Most chunks per call: keeps byte counts and grid sizes far from overflow
// (2^32 chunks of 2048 bits are 1 TiB, beyond any device's memory).
constexpr size_t kMaxChunks = (size_t)1 << 32;

// Host-side fault injection for tests: true when the environment variable
// PMK_INJECT_FAULT names `site`.  The *_host calls consult it right after
// they queue the copy of the caller's input ("after_copy") and then fail as a
// failed launch would, so a test can check that an error path leaves no
// copy of a caller's buffer in flight.  Nothing on the GPU faults.
bool fault_injected(const char *site);

// Exponent schedule for left-to-right sliding-window exponentiation.
// steps[0] = index of the first odd power (a load, no squaring);
// steps[i>0] = (nsq << 8) | idx : nsq squarings, then a multiply by the odd
// power table entry idx (x^(2 idx + 1)); idx = 0xFF means no multiply.
struct Schedule {
  std::vector<uint32_t> steps;
  uint32_t maxidx = 0;  // table entries 0..maxidx are needed
};

// Odd-power tables of the exponentiation kernels: the full table holds 16
// odd powers (windows up to 5 bits), the small one 8 (windows up to 4 bits)
// and takes half the shared memory, so more instances fit on an SM.  Every
// key carries one schedule set per table size, index kTableFull or
// kTableSmall.
enum : int { kTableFull = 0, kTableSmall = 1 };
constexpr uint32_t kWindowFull = 5, kWindowSmall = 4;
constexpr uint32_t window_of(int table) { return table == kTableSmall ? kWindowSmall : kWindowFull; }


// Most primes of one modulus (multi-prime RSA, Section 2.1).
constexpr int kMaxPrimes = 4;

// Joint schedule of two exponents (Straus / Shamir simultaneous
// exponentiation with interleaved sliding windows of width <= 4), for
// A^eA B^eB in one squaring chain.  steps[i] = (nsq << 16) | (ia << 8) | ib:
// nsq squarings, then multiplies by A's odd power ia and B's odd power ib
// (0xFF: none); steps[0] has nsq = 0 and loads instead of multiplying.
// Odd powers: A^(2 ia + 1), ia <= maxa <= 7, and likewise for B.
struct Schedule2 {
  std::vector<uint32_t> steps;
  uint32_t maxa = 0, maxb = 0;
};

// One key pair on the host, 32-bit little-endian limbs.  A key has b >= 2
// primes r_0 .. r_{b-1} of h = s / b limbs each; p = r_0, q = r_1.
struct HostKey {
  uint32_t nprimes = 2;
  std::vector<uint32_t> N, d, p, q, dp, dq, qinv;  // N, d: s limbs; the rest h
  std::vector<uint32_t> pr[kMaxPrimes], dpr[kMaxPrimes];  // r_i and d mod (r_i - 1)
  // Garner coefficients (exported with the key): coef_0 = qinv = r_1^-1 mod
  // r_0, coef_1 = 0, coef_i = (r_0 ... r_{i-1})^-1 mod r_i.
  std::vector<uint32_t> coef[kMaxPrimes];
  // CRT recombination rows, s limbs: c_i R mod N with
  // c_i = (N / r_i) ((N / r_i)^-1 mod r_i).
  std::vector<uint32_t> crt_sum[kMaxPrimes];
  // Montgomery data, R = 2^(32 s) for N and R_h = 2^(32 h) for the primes.
  uint32_t n0 = 0, n0h[kMaxPrimes] = {};               // -M^-1 mod 2^32
  std::vector<uint32_t> R2;                            // R^2 mod N
  std::vector<uint32_t> R2h[kMaxPrimes], R3h[kMaxPrimes];  // R_h^2, R_h^3 mod r_i
  // Exponent schedules per table size (kTableFull, kTableSmall): e, d,
  // d mod (r_i - 1) and r_i - 2 (Fermat inverses mod r_i).
  Schedule sched_e[2], sched_d[2], sched_h[2][kMaxPrimes], sched_hinv[2][kMaxPrimes];
  // Blinded CRT decryption: c*^(d_i) c_r^(r_i - 1 - d_i) mod r_i
  // = (c* c_r^-1)^d mod r_i, jointly.
  Schedule2 sched_blind[kMaxPrimes];
};

// Device view of one key (pointers into the key set's device blob).
struct KeyDev {
  // Schedules (steps, step count, highest table entry) per table size,
  // [kTableFull] or [kTableSmall].
  const uint32_t *N;
  const uint32_t *R2;
  const uint32_t *sched_e[2], *sched_d[2];
  const uint32_t *P[kMaxPrimes];
  const uint32_t *R2h[kMaxPrimes];
  const uint32_t *R3h[kMaxPrimes];
  const uint32_t *sched_h[2][kMaxPrimes], *sched_hinv[2][kMaxPrimes];
  const uint32_t *crt_sum[kMaxPrimes];  // c_i R mod N (s limbs)
  const uint32_t *sched_blind[kMaxPrimes];
  const uint32_t *e_limbs, *d_limbs;  // e (2 limbs) and d (s limbs), for the thread-per-chunk baseline
  uint32_t nprimes;
  uint32_t n0, n0h[kMaxPrimes];
  uint32_t nsteps_e[2], nsteps_d[2], nsteps_h[2][kMaxPrimes], nsteps_hinv[2][kMaxPrimes];
  uint32_t maxidx_e[2], maxidx_d[2], maxidx_h[2][kMaxPrimes], maxidx_hinv[2][kMaxPrimes];
  uint32_t nsteps_blind[kMaxPrimes], maxa_blind[kMaxPrimes], maxb_blind[kMaxPrimes];
};

// One unit of work of the persistent batch kernels: up to 32 / TPI chunks
// (first + i * stride, i < count) of one key, in one mode.
struct BatchTask {
  const KeyDev *key;
  const uint32_t *in;
  uint32_t *out;
  long long first, stride;
  int count;
  int mode;  // 0 encrypt, 1 full-d decrypt, 2 + i: CRT residue mod prime r_i
};

// Host keygen (keygen.cpp).
int host_keygen(uint32_t K, uint32_t nbits, uint64_t e, uint64_t seed, std::vector<HostKey> &out);
int host_keygen_mp(uint32_t K, uint32_t nbits, uint32_t nprimes, uint64_t e, uint64_t seed, std::vector<HostKey> &out);
bool valid_multiprime(uint32_t nbits, uint32_t nprimes);
int host_from_primes(uint32_t nbits, uint64_t e, const uint32_t *p, const uint32_t *q, HostKey &out);
int host_from_primes_mp(uint32_t nbits, uint32_t nprimes, uint64_t e, const uint32_t *primes, HostKey &out);
Schedule make_schedule(const uint32_t *exp, int nlimbs, uint32_t max_window = kWindowFull);
Schedule2 make_schedule2(const uint32_t *expa, const uint32_t *expb, int nlimbs);

// Kernel launchers (kernels_*.cu).  All return PMK_* codes.
enum class ExpMode : int { kEncrypt = 0, kDecrypt = 1, kCrtHalf = 2, kCrtInverse = 3 };
int launch_split(uint32_t nbits, const uint8_t *msg, size_t len, uint32_t *chunks, size_t n, cudaStream_t st);
int launch_join(uint32_t nbits, const uint32_t *chunks, size_t n, uint8_t *msg, size_t len, cudaStream_t st);
// Flags chunks >= their key's modulus (kStatusRange); with key_idx, the key
// of chunk t is key_idx[t], and an index >= K sets kStatusKeyIndex instead.
int launch_range_check(const KeyDev *keys, uint32_t K, uint32_t s, const uint32_t *in, size_t n,
                       uint32_t *status, cudaStream_t st, const uint32_t *key_idx = nullptr);
// Key groups for explicit key indices (key_idx[t] = key of chunk t): builds
// in `table` (key_groups_words(n, K) words) the padded segment offsets
// poff[0..K] followed by the slot table, chunks of key k in slots
// [poff[k], poff[k + 1]).  Indices >= K set kStatusKeyIndex in *status and
// their chunks get no slot.  K <= 16383.
// Each key's segment is padded to a multiple of `align` slots (a power of
// two, 1 .. kGroupAlign): the largest instances-per-block of the kernels
// that will read the table, so that a block never straddles two keys and a
// key has at most one partly filled block per kernel.
size_t key_groups_words(size_t n, uint32_t K);
int launch_key_groups(const uint32_t *key_idx, size_t n, uint32_t K, uint32_t align, uint32_t *table,
                      uint32_t *status, cudaStream_t st);

// Launch geometry of an exponentiation kernel: lanes per instance, Montgomery
// form (0 = one carry chain per lane, 1 = independent columns) and the
// odd-power table size (kTableFull or kTableSmall; a geometry compiled only
// with the full table runs with it).
struct KernelConfig {
  uint32_t tpi = 0, form = 0;
  int table = kTableFull;
};
// Instances per block of the exponentiation kernel of a geometry, and of the
// CRT recombination at a full width (0 if not built): the alignment a key
// group table needs for them.
uint32_t modexp_block_instances(uint32_t limbs, KernelConfig cfg, bool crt);
uint32_t crt_sum_block_instances(uint32_t limbs);
// CRT modes run `parts` residues per chunk (the key's prime count) over
// `limbs` = s / parts limbs each; residue i of chunk t goes to out[t][i * limbs].
// With `groups` (a table of launch_key_groups built with alignment
// groups_align) chunks are taken by key group instead of round robin.
int launch_modexp(ExpMode mode, uint32_t limbs, KernelConfig cfg, const KeyDev *keys, uint32_t K, const uint32_t *in,
                  uint32_t *out, size_t n, cudaStream_t st, uint32_t parts = 2, const uint32_t *groups = nullptr,
                  uint32_t groups_align = kGroupAlign);
// CRT recombination of `parts` residues per chunk (limbs / parts limbs
// each) in place at full width `limbs`: out[t] holds the residues and
// receives the value mod N.
int launch_crt_sum(uint32_t limbs, uint32_t parts, const KeyDev *keys, uint32_t K, uint32_t *out, size_t n,
                   cudaStream_t st, uint32_t *status_if_zero_residue = nullptr, const uint32_t *groups = nullptr,
                   uint32_t groups_align = kGroupAlign);
// Fused blinded CRT decryption: out[t][i] = c*[t]^(d_i) c_r[t]^(r_i - 1 - d_i)
// mod r_i for each of the key's `parts` primes (prime_limbs limbs each); the
// residues of (c* c_r^-1)^d, to be recombined by launch_crt_sum.  A c_r
// divisible by a prime sets kStatusNotInvertible in *status.
int launch_blind_crt(uint32_t prime_limbs, uint32_t parts, const KeyDev *keys, uint32_t K, const uint32_t *cstar,
                     const uint32_t *cr, uint32_t *out, size_t n, cudaStream_t st, uint32_t *status);
bool blind_crt_built(uint32_t prime_limbs);
// out[t] = a[t] * b[t] mod N_{t mod K} (full width; out may alias a or b)
int launch_mulmod(uint32_t limbs, const KeyDev *keys, uint32_t K, const uint32_t *a, const uint32_t *b, uint32_t *out,
                  size_t n, cudaStream_t st);
bool modexp_built(uint32_t limbs, KernelConfig cfg, bool crt);
// Whether that geometry is also compiled with the small odd-power table.
bool modexp_small_table_built(uint32_t limbs, KernelConfig cfg, bool crt);
// The plain thread-per-chunk, binary-exponent kernel (a measured baseline; 32 or 64 limbs).
int launch_modexp_naive(bool enc, uint32_t limbs, const KeyDev *keys, uint32_t K, const uint32_t *in, uint32_t *out,
                        size_t n, cudaStream_t st);
KernelConfig default_config(uint32_t limbs, bool crt);  // tpi == 0: limb count not built
int list_configs(uint32_t limbs, bool crt, KernelConfig *out, int max);
// Persistent batch kernel for (limbs, cfg, crt): `blocks` x 128 threads
// drain tasks[0..ntasks) through *counter (which must start at zero).
int launch_modexp_tasks(uint32_t limbs, KernelConfig cfg, bool crt, const BatchTask *tasks, int ntasks, int *counter,
                        int blocks, cudaStream_t st);
// Resident blocks per SM of that kernel (0 if not built).
int modexp_tasks_blocks_per_sm(uint32_t limbs, KernelConfig cfg, bool crt);
// Exponentiations the whole GPU holds at once in that geometry (0 if not built).
long long modexp_resident_instances(uint32_t limbs, KernelConfig cfg, bool crt);
int measure_int_peak(double *macs_per_clk_per_sm, double *sm_mhz, int *num_sms);
// Raise a kernel's dynamic shared-memory limit to `bytes`, once per (kernel, device).
int configure_smem(const void *fn, size_t bytes);
int measure_imad_peak(double *mad_lo_per_clk_per_sm, double *sm_mhz, int *num_sms);

}  // namespace pmk

// Key set: host copy and device-resident tables (opaque in the C ABI).
struct pmk_keyset {
  int device = 0;
  uint32_t K = 0, nbits = 0;
  uint32_t nprimes = 2;                    // primes per modulus
  uint64_t e = 0;
  std::vector<pmk::HostKey> keys;
  uint32_t *d_blob = nullptr;              // every key's limbs and schedules
  pmk::KeyDev *d_keys = nullptr;           // K device key views into d_blob
};

namespace pmk {
// A grow-only device buffer owned by a context, allocated and freed in
// stream order (cudaMallocAsync / cudaFreeAsync).  `last_use` is recorded
// on the stream of the last call that used it; the next call waits on it on
// its own stream before reusing, growing or freeing the buffer, so staging
// never overlaps work still in flight on another stream.
struct Staging {
  void *ptr = nullptr;
  size_t cap = 0;
  cudaEvent_t last_use = nullptr;
};
}  // namespace pmk

namespace pmk {
// Default direct-launch limit of batch planning (see batch_plan.h).
constexpr size_t kDirectMaxJobs = 256;
}  // namespace pmk

// Context: one device, its status record, staging and kernel geometry choices.
struct pmk_ctx {
  int device = 0;
  uint32_t *d_status = nullptr;            // status record: error bits, smallest failing chunk
  pmk::Staging msg, a, b;                  // staging of the *_host calls and the blinded CRT path
  pmk::Staging grp;                        // key-group table of calls with explicit key indices
  std::map<uint32_t, pmk::KernelConfig> cfg;  // (limbs << 1 | crt) -> kernel geometry override
  std::map<uint32_t, int> table;              // (limbs << 1 | crt) -> odd-power table size override
  size_t batch_direct_max = pmk::kDirectMaxJobs;  // pmk_set_batch_direct_max
};
