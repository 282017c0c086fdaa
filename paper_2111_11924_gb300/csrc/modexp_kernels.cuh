// Exponentiation kernels built on modexp_core.cuh, and the table that maps a
// (mode, limb count, threads per instance) triple to an instantiation.
#pragma once

#include "modexp_core.cuh"

namespace pmk {
namespace dev {

// Grid: blockIdx.y selects the key (full width) or key * 2 + half (CRT);
// blockIdx.x * IPB + instance slot selects the j-th chunk of that key, chunk
// t = key + j K.  Every block therefore serves one key: schedules, modulus and
// control flow are uniform across it.
//
// FULL: out[t] = in[t]^E mod N_key, E = e (sel != 0) or d, S = nbits / 32.
// CRT:  out[t][half] = in[t]^E mod (p | q) over S = nbits / 64 limbs, with
//       E = d_p | d_q (sel == 0), or p - 2 | q - 2 (sel != 0: inverses mod p,
//       q by Fermat's little theorem), 
//       input reduced via in mod p = hi R + lo -> MontMul(hi, R^3) +
//       MontMul(lo, R^2) = in R mod p.  Garner combines the halves afterwards.
template <int S, int TPI, bool CRT, int FORM>
__global__ void __launch_bounds__(kThreads) k_modexp(const KeyDev *__restrict__ keys, uint32_t K,
                                                     const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                                                     long long n, int sel) {
  constexpr int L = S / TPI;
  constexpr int IPB = kThreads / TPI;
  constexpr int ROW = Layout<S>::kRow;
  constexpr int INST = Layout<S>::kInst;
  constexpr int W = CRT ? 2 * S : S;  // limbs per chunk in memory
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t *sR2 = smem, *sOne = smem + ROW, *sR3 = smem + 2 * ROW;
  const uint32_t r = threadIdx.x % TPI, g = threadIdx.x / TPI;
  uint32_t *tbl = smem + Layout<S>::kConstRows * ROW + g * INST;
  uint32_t *ybuf = tbl + kTableMax * ROW;

  const uint32_t key = CRT ? blockIdx.y >> 1 : blockIdx.y;
  const uint32_t half = CRT ? blockIdx.y & 1 : 0;
  const long long first = key + (long long)blockIdx.x * IPB * K;
  if (first >= n) return;  // block-uniform: no instance of this block has a chunk
  const KeyDev &kd = keys[key];
  const uint32_t *M = CRT ? kd.P[half] : kd.N;
  const uint32_t *R2 = CRT ? kd.R2h[half] : kd.R2;
  const uint32_t *sched = CRT ? (sel ? kd.sched_hinv[half] : kd.sched_h[half]) : (sel ? kd.sched_e : kd.sched_d);
  const uint32_t nsteps = CRT ? (sel ? kd.nsteps_hinv[half] : kd.nsteps_h[half]) : (sel ? kd.nsteps_e : kd.nsteps_d);
  const uint32_t maxidx = CRT ? (sel ? kd.maxidx_hinv[half] : kd.maxidx_h[half]) : (sel ? kd.maxidx_e : kd.maxidx_d);
  const uint32_t n0 = CRT ? kd.n0h[half] : kd.n0;

  for (int i = threadIdx.x; i < S; i += kThreads) {
    sR2[i] = __ldg(R2 + i);
    sOne[i] = (i == 0);
    if (CRT) sR3[i] = __ldg(kd.R3h[half] + i);
  }
  __syncthreads();

  const long long t = first + (long long)g * K;
  const bool active = t < n;
  uint32_t nn[L], a[L];
  load_slice_global<L>(nn, M, r);
  if (!CRT) {
    if (active) {
      load_slice_global<L>(a, in + t * W, r);
    } else {
#pragma unroll
      for (int j = 0; j < L; j++) a[j] = 0;
    }
    mont<S, TPI, FORM>(a, sR2, nn, n0, r);  // x R mod N
  } else {
    uint32_t lo[L];
    if (active) {
      load_slice_global<L>(lo, in + t * W, r);
      load_slice_global<L>(a, in + t * W + S, r);
    } else {
#pragma unroll
      for (int j = 0; j < L; j++) lo[j] = a[j] = 0;
    }
    mont<S, TPI, FORM>(a, sR3, nn, n0, r);   // hi R^2 mod p
    mont<S, TPI, FORM>(lo, sR2, nn, n0, r);  // lo R mod p
    mod_add<L, TPI>(a, lo, nn, r);         // (hi R + lo) R mod p
  }
  exp_window<S, TPI, FORM>(a, tbl, ybuf, sched, nsteps, maxidx, nn, n0, r);
  mont<S, TPI, FORM>(a, sOne, nn, n0, r);  // leave the Montgomery domain
  if (active) {
    uint32_t *o = out + t * W + (CRT ? half * S : 0) + r * L;
    if constexpr (L % 4 == 0) {
#pragma unroll
      for (int j = 0; j < L; j += 4) *reinterpret_cast<uint4 *>(o + j) = make_uint4(a[j], a[j + 1], a[j + 2], a[j + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < L; j++) o[j] = a[j];
    }
  }
}

// Persistent form for batches: each warp repeatedly takes the next task from
// a device counter.  A task is up to 32 / TPI chunks of one key of one job
// (chunk first + i * stride), in one mode.  Keys differ from warp to warp, so
// the constant rows (R^2, 1, R^3) live in each warp's own shared-memory area.
template <int S, int TPI, bool CRT, int FORM>
__global__ void __launch_bounds__(kThreads) k_modexp_tasks(const BatchTask *__restrict__ tasks, int ntasks,
                                                           int *__restrict__ counter) {
  constexpr int L = S / TPI;
  constexpr int IPW = 32 / TPI;
  constexpr int ROW = Layout<S>::kRow;
  constexpr int INST = Layout<S>::kInst;
  constexpr int W = CRT ? 2 * S : S;
  constexpr int WAREA = Layout<S>::kConstRows * ROW + IPW * INST;
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t lane = threadIdx.x & 31, r = lane % TPI, g = lane / TPI;
  uint32_t *wbase = smem + (threadIdx.x / 32) * WAREA;
  uint32_t *sR2 = wbase, *sOne = wbase + ROW, *sR3 = wbase + 2 * ROW;
  uint32_t *tbl = wbase + Layout<S>::kConstRows * ROW + g * INST;
  uint32_t *ybuf = tbl + kTableMax * ROW;
  for (;;) {
    int ti = 0;
    if (lane == 0) ti = atomicAdd(counter, 1);
    ti = __shfl_sync(kFull, ti, 0);
    if (ti >= ntasks) break;
    const BatchTask tk = tasks[ti];
    const KeyDev &kd = *tk.key;
    const int half = tk.mode == 3 ? 1 : 0;
    const bool enc = tk.mode == 0;
    const uint32_t *M = CRT ? kd.P[half] : kd.N;
    const uint32_t *R2 = CRT ? kd.R2h[half] : kd.R2;
    const uint32_t *sched = CRT ? kd.sched_h[half] : (enc ? kd.sched_e : kd.sched_d);
    const uint32_t nsteps = CRT ? kd.nsteps_h[half] : (enc ? kd.nsteps_e : kd.nsteps_d);
    const uint32_t maxidx = CRT ? kd.maxidx_h[half] : (enc ? kd.maxidx_e : kd.maxidx_d);
    const uint32_t n0 = CRT ? kd.n0h[half] : kd.n0;
    __syncwarp();  // the previous task's reads of the constant rows are done
    for (int i = lane; i < S; i += 32) {
      sR2[i] = __ldg(R2 + i);
      sOne[i] = (i == 0);
      if (CRT) sR3[i] = __ldg(kd.R3h[half] + i);
    }
    __syncwarp();
    const bool active = (int)g < tk.count;
    const long long t = tk.first + (long long)g * tk.stride;
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
      uint32_t lo[L];
      if (active) {
        load_slice_global<L>(lo, tk.in + t * W, r);
        load_slice_global<L>(a, tk.in + t * W + S, r);
      } else {
#pragma unroll
        for (int j = 0; j < L; j++) lo[j] = a[j] = 0;
      }
      mont<S, TPI, FORM>(a, sR3, nn, n0, r);
      mont<S, TPI, FORM>(lo, sR2, nn, n0, r);
      mod_add<L, TPI>(a, lo, nn, r);
    }
    exp_window<S, TPI, FORM>(a, tbl, ybuf, sched, nsteps, maxidx, nn, n0, r);
    mont<S, TPI, FORM>(a, sOne, nn, n0, r);
    if (active) {
      uint32_t *o = tk.out + t * W + (CRT ? half * S : 0) + r * L;
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

template <int S>
constexpr size_t modexp_smem_bytes(int tpi) {
  return sizeof(uint32_t) * ((size_t)Layout<S>::kConstRows * Layout<S>::kRow + (size_t)(kThreads / tpi) * Layout<S>::kInst);
}

}  // namespace dev

// One compiled instantiation: limb count, lanes per instance, CRT or full
// width, Montgomery form (dev::kChain / dev::kCols); the one-launch-per-call
// kernel and the persistent batch kernel with their shared-memory sizes.
struct ModexpEntry {
  int limbs, tpi;
  bool crt;
  int form;
  const void *fn;
  size_t smem;
  const void *fn_tasks;
  size_t smem_tasks;
};

template <int S, int TPI, bool CRT, int FORM>
ModexpEntry make_entry() {
  constexpr size_t warp_area = (size_t)dev::Layout<S>::kConstRows * dev::Layout<S>::kRow +
                               (size_t)(32 / TPI) * dev::Layout<S>::kInst;
  return ModexpEntry{S, TPI, CRT, FORM, reinterpret_cast<const void *>(&dev::k_modexp<S, TPI, CRT, FORM>),
                     dev::modexp_smem_bytes<S>(TPI),
                     reinterpret_cast<const void *>(&dev::k_modexp_tasks<S, TPI, CRT, FORM>),
                     sizeof(uint32_t) * warp_area * (dev::kThreads / 32)};
}

// Instantiation lists live in separate translation units (compiled in parallel).
const ModexpEntry *modexp_entries_full(int *count);
const ModexpEntry *modexp_entries_crt(int *count);
const ModexpEntry *modexp_entries_wide(int *count);  // 6144/8192-bit full width, 3072/4096-bit CRT halves

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

}  // namespace pmk
