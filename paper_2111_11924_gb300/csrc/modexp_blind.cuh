// Blinded CRT decryption in one pass per prime (Algorithm 1 "Decryption"
// with the random matrix R, in the Section 2.1 CRT form).
//
// Algorithm 1 recovers m' = m* r'^-1 with m* = c*^d and r' = c_r^d (mod N).
// Modulo each prime r_i of N, and for c_r a unit mod r_i, that residue is
//     (c* c_r^-1)^d = c*^(d_i) * c_r^(r_i - 1 - d_i)   (mod r_i),
// with d_i = d mod (r_i - 1) (Fermat: c_r^(r_i - 1) = 1).  Both powers run
// in one squaring chain (simultaneous exponentiation with interleaved
// sliding windows, Straus / Shamir): about n/b squarings plus the windows
// of the two exponents, instead of a Fermat inversion, a product and a
// second exponentiation.  The residues are recombined by k_crt_sum.
#pragma once

#include "modexp_grid.cuh"

namespace pmk {
namespace dev {

static_assert(kTableMax >= 16, "the joint tables use rows 0-7 (A) and 8-15 (B)");

// a <- A^eA B^eB in Montgomery form.  On entry rows 0 and 8 of tbl hold A
// and B (Montgomery form, this instance); tbl gets A's odd powers in rows
// 0..maxa and B's in rows 8..8+maxb; ybuf is the squaring buffer.  sched is
// a Schedule2 (block-uniform).
template <int S, int TPI, int FORM>
__device__ __forceinline__ void exp2_window(uint32_t (&a)[S / TPI], uint32_t *tbl, uint32_t *ybuf,
                                            const uint32_t *__restrict__ sched, uint32_t nsteps, uint32_t maxa,
                                            uint32_t maxb, const uint32_t (&nn)[S / TPI], uint32_t n0, uint32_t r) {
  constexpr int L = S / TPI;
  constexpr int ROW = Layout<S>::kRow;
#pragma unroll 1
  for (int which = 0; which < 2; which++) {  // odd powers of A, then of B
    uint32_t *base = tbl + which * 8 * ROW;
    const uint32_t maxi = which ? maxb : maxa;
    if (maxi == 0) continue;
    load_slice<L>(a, base, r);
    __syncwarp();
    store_slice<L>(ybuf, a, r);
    __syncwarp();
    mont<S, TPI, FORM>(a, ybuf, nn, n0, r);  // X^2
    __syncwarp();
    store_slice<L>(ybuf, a, r);
    load_slice<L>(a, base, r);
    __syncwarp();
#pragma unroll 1
    for (uint32_t k = 1; k <= maxi; k++) {  // row k = X^(2k+1)
      mont<S, TPI, FORM>(a, ybuf, nn, n0, r);
      store_slice<L>(base + k * ROW, a, r);
    }
    __syncwarp();
  }
  __syncwarp();  // rows 0 and 8, stored by the caller, are read whole below
  const uint32_t s0 = __ldg(sched);
  const uint32_t ia0 = (s0 >> 8) & 0xffu, ib0 = s0 & 0xffu;
  if (ia0 != 0xffu) {
    load_slice<L>(a, tbl + ia0 * ROW, r);
    if (ib0 != 0xffu) mont<S, TPI, FORM>(a, tbl + (8 + ib0) * ROW, nn, n0, r);
  } else {
    load_slice<L>(a, tbl + (8 + ib0) * ROW, r);
  }
#pragma unroll 1
  for (uint32_t si = 1; si < nsteps; si++) {
    const uint32_t step = __ldg(sched + si);
    const uint32_t nsq = step >> 16, ia = (step >> 8) & 0xffu, ib = step & 0xffu;
#pragma unroll 1
    for (uint32_t k = 0; k < nsq; k++) {
      __syncwarp();
      store_slice<L>(ybuf, a, r);
      __syncwarp();
      mont<S, TPI, FORM>(a, ybuf, nn, n0, r);
    }
    if (ia != 0xffu) mont<S, TPI, FORM>(a, tbl + ia * ROW, nn, n0, r);
    if (ib != 0xffu) mont<S, TPI, FORM>(a, tbl + (8 + ib) * ROW, nn, n0, r);
  }
}

// out[t][i] = c*[t]^(d_i) c_r[t]^(r_i - 1 - d_i) mod r_i for every prime r_i
// of the chunk's key (grid as the CRT mode of k_modexp: blockIdx.y = key *
// parts + i).  With `status`, a c_r divisible by r_i (no inverse mod N)
// sets kStatusNotInvertible.
template <int S, int TPI, int FORM, int NT>
__global__ void __launch_bounds__(NT) k_blind_crt(const KeyDev *__restrict__ keys, uint32_t K,
                                                  const uint32_t *__restrict__ cstar, const uint32_t *__restrict__ cr,
                                                  uint32_t *__restrict__ out, long long n, int parts,
                                                  uint32_t *__restrict__ status) {
  constexpr int L = S / TPI;
  constexpr int IPB = NT / TPI;
  constexpr int ROW = Layout<S>::kRow;
  constexpr int INST = Layout<S>::kInst;
  const int W = parts * S;
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t *sR2 = smem, *sOne = smem + ROW, *sR3 = smem + 2 * ROW;
  const uint32_t r = threadIdx.x % TPI, g = threadIdx.x / TPI;
  uint32_t *tbl = smem + Layout<S>::kConstRows * ROW + g * INST;
  uint32_t *ybuf = tbl + kTableMax * ROW;

  const uint32_t key = blockIdx.y / (uint32_t)parts;
  const uint32_t prime = blockIdx.y % (uint32_t)parts;
  const long long first = key + (long long)blockIdx.x * IPB * K;
  if (first >= n) return;  // block-uniform
  const KeyDev &kd = keys[key];
  for (int i = threadIdx.x; i < S; i += NT) {
    sR2[i] = __ldg(kd.R2h[prime] + i);
    sOne[i] = (i == 0);
    sR3[i] = __ldg(kd.R3h[prime] + i);
  }
  __syncthreads();
  // After the barrier the warps are independent: a warp whose instances all
  // lie past the last chunk (the tail block of a key) leaves.
  if (first + (long long)((threadIdx.x / 32) * (32 / TPI)) * K >= n) return;

  const long long t = first + (long long)g * K;
  const bool active = t < n;
  const uint32_t n0 = kd.n0h[prime];
  uint32_t nn[L], a[L];
  load_slice_global<L>(nn, kd.P[prime], r);
  crt_input<S, TPI, FORM>(a, cstar + t * W, active, parts, sR2, sR3, nn, n0, r);  // A = c* R mod r_i
  store_slice<L>(tbl, a, r);
  crt_input<S, TPI, FORM>(a, cr + t * W, active, parts, sR2, sR3, nn, n0, r);     // B = c_r R mod r_i
  uint32_t any = 0;
#pragma unroll
  for (int j = 0; j < L; j++) any |= a[j];
  if constexpr (TPI > 1) {
#pragma unroll
    for (int o = 1; o < TPI; o <<= 1) any |= __shfl_xor_sync(kFull, any, o, TPI);
  }
  if (status && active && r == 0 && any == 0) report(status, kStatusNotInvertible, t);
  store_slice<L>(tbl + 8 * ROW, a, r);
  exp2_window<S, TPI, FORM>(a, tbl, ybuf, kd.sched_blind[prime], kd.nsteps_blind[prime], kd.maxa_blind[prime],
                            kd.maxb_blind[prime], nn, n0, r);
  mont<S, TPI, FORM>(a, sOne, nn, n0, r);  // leave the Montgomery domain
  if (active) {
    uint32_t *o = out + t * W + prime * S + r * L;
#pragma unroll
    for (int j = 0; j < L; j++) o[j] = a[j];
  }
}

}  // namespace dev
}  // namespace pmk
