// Exponentiation kernels built on modexp_core.cuh, and the table that maps a
// (mode, limb count, threads per instance) triple to an instantiation.
#pragma once

#include "modexp_grid.cuh"

namespace pmk {
namespace dev {

// The value 1 as a row of limbs, for leaving the Montgomery domain.
static __device__ __align__(16) uint32_t g_one_row[256] = {1u};

// Persistent form for batches: each warp repeatedly takes the next task from
// a device counter.  A task is up to 32 / TPI chunks of one key of one job
// (chunk first + i * stride), in one mode (CRT residue i of a key with
// nprimes primes: mode 2 + i).  Keys differ from warp to warp, so the rows
// used once or twice per exponentiation (R^2, R^3, 1) are read from global
// memory (the key blob, L1-cached) instead of shared memory; a block then
// needs only its instances' tables, as many blocks fit per SM as for
// k_modexp.
template <int S, int TPI, bool CRT, int FORM, int TABLE = kTableFull>
__global__ void __launch_bounds__(kThreads) k_modexp_tasks(const BatchTask *__restrict__ tasks, int ntasks,
                                                           int *__restrict__ counter) {
  constexpr int L = S / TPI;
  constexpr int IPW = 32 / TPI;
  constexpr int ROW = Layout<S>::kRow;
  constexpr int ROWS = table_rows(TABLE);
  constexpr int INST = Layout<S>::inst(ROWS);
  constexpr int WAREA = IPW * INST;
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t lane = threadIdx.x & 31, r = lane % TPI, g = lane / TPI;
  uint32_t *wbase = smem + (threadIdx.x / 32) * WAREA;
  uint32_t *tbl = wbase + g * INST;
  uint32_t *ybuf = tbl + ROWS * ROW;
  for (;;) {
    int ti = 0;
    if (lane == 0) ti = atomicAdd(counter, 1);
    ti = __shfl_sync(kFull, ti, 0);
    if (ti >= ntasks) break;
    const BatchTask tk = tasks[ti];
    const KeyDev &kd = *tk.key;
    const int prime = tk.mode >= 2 ? tk.mode - 2 : 0;
    const bool enc = tk.mode == 0;
    const int parts = CRT ? (int)kd.nprimes : 1;
    const int W = parts * S;
    const uint32_t *M = CRT ? kd.P[prime] : kd.N;
    const uint32_t *R2 = CRT ? kd.R2h[prime] : kd.R2;
    const uint32_t *sched = CRT ? kd.sched_h[TABLE][prime] : (enc ? kd.sched_e[TABLE] : kd.sched_d[TABLE]);
    const uint32_t nsteps = CRT ? kd.nsteps_h[TABLE][prime] : (enc ? kd.nsteps_e[TABLE] : kd.nsteps_d[TABLE]);
    const uint32_t maxidx = CRT ? kd.maxidx_h[TABLE][prime] : (enc ? kd.maxidx_e[TABLE] : kd.maxidx_d[TABLE]);
    const uint32_t n0 = CRT ? kd.n0h[prime] : kd.n0;
    const uint32_t *sR2 = R2, *sR3 = CRT ? kd.R3h[prime] : R2, *sOne = g_one_row;
    const bool active = (int)g < tk.count;
    const long long t = tk.first + (long long)g * tk.stride;
    // The output address is formed before the exponentiation, so that only
    // this pointer (not the task's fields) stays live across it.
    uint32_t *const o = active ? tk.out + t * W + (CRT ? prime * S : 0) + r * L : nullptr;
    uint32_t nn[L], a[L];
    load_slice_global<L>(nn, M, r);
    if (!CRT) {
      if (active) {
        load_slice_global<L>(a, tk.in + t * W, r);
      } else {
#pragma unroll
        for (int j = 0; j < L; j++) a[j] = 0;
      }
      mont<S, TPI, FORM>(a, sR2, nn, n0, r);
    } else {
      crt_input<S, TPI, FORM>(a, tk.in + t * W, active, parts, sR2, sR3, nn, n0, r);
    }
    exp_window<S, TPI, FORM>(a, tbl, ybuf, sched, nsteps, maxidx, nn, n0, r);
    mont<S, TPI, FORM>(a, sOne, nn, n0, r);
    if (o) {
      if constexpr (L % 4 == 0) {
#pragma unroll
        for (int j = 0; j < L; j += 4) *reinterpret_cast<uint4 *>(o + j) = make_uint4(a[j], a[j + 1], a[j + 2], a[j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < L; j++) o[j] = a[j];
      }
    }
  }
}

// out[t] = a[t] b[t] mod N_key: two Montgomery products, a b R^-1 and then
// (a b R^-1) R^2 R^-1.  Same grid mapping as k_modexp; b goes through shared
// memory as the broadcast operand.
template <int S, int TPI>
__global__ void __launch_bounds__(kThreads) k_mulmod(const KeyDev *__restrict__ keys, uint32_t K,
                                                     const uint32_t *a_in, const uint32_t *b_in, uint32_t *out,
                                                     long long n) {
  constexpr int L = S / TPI;
  constexpr int IPB = kThreads / TPI;
  constexpr int ROW = Layout<S>::kRow;
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t r = threadIdx.x % TPI, g = threadIdx.x / TPI;
  uint32_t *sR2 = smem, *yrow = smem + (1 + g) * ROW;
  const uint32_t key = blockIdx.y;
  const long long first = key + (long long)blockIdx.x * IPB * K;
  if (first >= n) return;
  const KeyDev &kd = keys[key];
  for (int i = threadIdx.x; i < S; i += kThreads) sR2[i] = __ldg(kd.R2 + i);
  const long long t = first + (long long)g * K;
  const bool active = t < n;
  uint32_t nn[L], a[L], b[L];
  load_slice_global<L>(nn, kd.N, r);
  if (active) {
    load_slice_global<L>(a, a_in + t * S, r);
    load_slice_global<L>(b, b_in + t * S, r);
  } else {
#pragma unroll
    for (int j = 0; j < L; j++) a[j] = b[j] = 0;
  }
  store_slice<L>(yrow, b, r);
  __syncthreads();
  mont<S, TPI, kChain>(a, yrow, nn, kd.n0, r);
  mont<S, TPI, kChain>(a, sR2, nn, kd.n0, r);
  if (active) {
    uint32_t *o = out + t * S + r * L;
#pragma unroll
    for (int j = 0; j < L; j++) o[j] = a[j];
  }
}

// CRT recombination at full width.  The congruences x = m_i mod r_i
// (i < B) have one solution below N = r_0 ... r_{B-1} (the Chinese remainder
// theorem, Section 2.1): x = sum_i m_i c_i mod N with c_i = (N / r_i) times
// ((N / r_i)^-1 mod r_i), since c_i = 1 mod r_i and 0 mod every other prime.
// Each term is one Montgomery product of the residue with the key's row
// c_i R mod N, so the kernel is B products and B modular additions per
// chunk.  In place: chunk t of `out` (S limbs) holds the B residues, S / B
// limbs each, and receives x.  Every lane has consumed its loads of the last
// residue before the group's shuffles inside that product, so the stores
// cannot overtake another lane's loads.  With `status`, a residue equal to
// zero (the input shares the prime r_i: no inverse exists) sets
// kStatusNotInvertible.  Grid as k_mulmod, or over key groups as k_modexp
// (block_chunks) when grp is given.
template <int S, int TPI>
__global__ void __launch_bounds__(kThreads) k_crt_sum(const KeyDev *__restrict__ keys, uint32_t K,
                                                      uint32_t *out, long long n, int B, uint32_t *status,
                                                      const uint32_t *__restrict__ grp) {
  constexpr int L = S / TPI;
  constexpr int IPB = kThreads / TPI;
  constexpr int ROW = Layout<S>::kRow;
  extern __shared__ __align__(16) uint32_t smem[];  // B rows: c_i R mod N
  const uint32_t r = threadIdx.x % TPI, g = threadIdx.x / TPI;
  const BlockChunks bc = block_chunks(grp, K, n, IPB, blockIdx.y);
  if (!bc.any) return;
  const KeyDev &kd = keys[bc.key];
  for (int i = threadIdx.x; i < B * S; i += kThreads) smem[(i / S) * ROW + i % S] = __ldg(kd.crt_sum[i / S] + i % S);
  __syncthreads();
  const long long t = slot_chunk(grp, K, n, bc, g);
  const bool active = t >= 0;
  const int H = S / B;
  uint32_t nn[L], acc[L], a[L];
  load_slice_global<L>(nn, kd.N, r);
#pragma unroll
  for (int j = 0; j < L; j++) acc[j] = 0;
  bool zero = false;
  for (int i = 0; i < B; i++) {
    uint32_t any = 0;
#pragma unroll
    for (int j = 0; j < L; j++) {  // residue i, zero-extended to S limbs
      const int limb = (int)r * L + j;
      a[j] = (active && limb < H) ? out[t * S + i * H + limb] : 0u;
      any |= a[j];
    }
    if constexpr (TPI > 1) {
#pragma unroll
      for (int o = 1; o < TPI; o <<= 1) any |= __shfl_xor_sync(kFull, any, o, TPI);
    }
    zero = zero || any == 0;
    mont<S, TPI, kChain>(a, smem + i * ROW, nn, kd.n0, r);  // m_i c_i mod N
    mod_add<L, TPI>(acc, a, nn, r);
  }
  if (active) {
    if (status && zero && r == 0) report(status, kStatusNotInvertible, t);
    uint32_t *o = out + t * S + r * L;
#pragma unroll
    for (int j = 0; j < L; j++) o[j] = acc[j];
  }
}

template <int S>
constexpr size_t modexp_smem_bytes(int tpi, int threads = kThreads, int table = kTableFull) {
  return sizeof(uint32_t) * ((size_t)Layout<S>::kConstRows * Layout<S>::kRow +
                             (size_t)(threads / tpi) * Layout<S>::inst(table_rows(table)));
}

}  // namespace dev

// One compiled instantiation: limb count, lanes per instance, CRT or full
// width, Montgomery form (dev::kChain / dev::kCols), odd-power table size
// (kTableFull / kTableSmall); the one-launch-per-call kernel (round robin,
// and its twin over key groups) and the persistent batch kernel with their
// shared-memory sizes.
struct ModexpEntry {
  int limbs, tpi;
  bool crt;
  int form;
  const void *fn;
  const void *fn_grp;  // fn over a key group table (same shared memory)
  size_t smem;
  const void *fn_tasks;
  size_t smem_tasks;
  int threads;  // block size of fn (fn_tasks always uses dev::kThreads)
  int table;
};

// NT: block size of the one-launch-per-call kernel.  64 for 32 limbs at 4
// lanes: a 128-thread block (32 instance tables, 78 KB) leaves two per SM
// and much shared memory unused, 64-thread blocks fit five (64 -> 80
// instances per SM): 3.4% faster CRT decryption at 2048 bits and 100 MiB.
// Other geometries measured no gain or a loss (64 limbs at 4 lanes: 12%
// slower at 1 MiB) and keep 128.
// RR_GRP: round-robin launches also take the key-group instantiation (the
// geometries where it measured faster; see k_modexp).  GRP_MINB: the
// key-group instantiation's minimum resident blocks per SM, where it differs
// from MINB (the geometries where it measured faster that way).
template <int S, int TPI, bool CRT, int FORM, int NT = dev::kThreads, int TABLE = kTableFull, int MINB = 0,
          bool RR_GRP = false, int GRP_MINB = MINB>
ModexpEntry make_entry() {
  constexpr size_t warp_area = (size_t)(32 / TPI) * dev::Layout<S>::inst(dev::table_rows(TABLE));
  return ModexpEntry{S,
                     TPI,
                     CRT,
                     FORM,
                     reinterpret_cast<const void *>(
                         &dev::k_modexp<S, TPI, CRT, FORM, NT, TABLE, RR_GRP ? GRP_MINB : MINB, RR_GRP>),
                     reinterpret_cast<const void *>(&dev::k_modexp<S, TPI, CRT, FORM, NT, TABLE, GRP_MINB, true>),
                     dev::modexp_smem_bytes<S>(TPI, NT, TABLE),
                     reinterpret_cast<const void *>(&dev::k_modexp_tasks<S, TPI, CRT, FORM, TABLE>),
                     sizeof(uint32_t) * warp_area * (dev::kThreads / 32),
                     NT,
                     TABLE};
}

// Instantiation lists live in separate translation units (compiled in parallel).
const ModexpEntry *modexp_entries_full(int *count);
const ModexpEntry *modexp_entries_crt(int *count);
const ModexpEntry *modexp_entries_wide(int *count);  // 6144/8192-bit full width, their CRT residues
const ModexpEntry *modexp_entries_latency(int *count);  // more lanes per instance for small batches
const ModexpEntry *modexp_entries_small(int *count);    // CRT residue kernels with the small table

// Modular multiplication kernels, one per full-width limb count.
struct MulmodEntry {
  int limbs, tpi;
  const void *fn;
  size_t smem;
};
template <int S, int TPI>
MulmodEntry make_mulmod() {
  return MulmodEntry{S, TPI, reinterpret_cast<const void *>(&dev::k_mulmod<S, TPI>),
                     sizeof(uint32_t) * (size_t)(1 + dev::kThreads / TPI) * dev::Layout<S>::kRow};
}
const MulmodEntry *mulmod_entries(int *count);

// CRT recombination kernels, one per full-width limb count (same geometries
// as the modular multiplication).
template <int S, int TPI>
MulmodEntry make_crt_sum() {
  return MulmodEntry{S, TPI, reinterpret_cast<const void *>(&dev::k_crt_sum<S, TPI>),
                     sizeof(uint32_t) * (size_t)kMaxPrimes * dev::Layout<S>::kRow};
}
const MulmodEntry *crt_sum_entries(int *count);

}  // namespace pmk
