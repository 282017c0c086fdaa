// The one-launch-per-call exponentiation kernel (encryption, full-d
// decryption, CRT residues) built on modexp_core.cuh.
#pragma once

#include "modexp_core.cuh"

namespace pmk {
namespace dev {

// The CRT input of one residue in Montgomery form: x = c R mod r for the
// chunk c = sum_j c_j R^j of `parts` S-limb pieces (R = 2^(32 S)), by Horner
// from the top piece: MontMul(c_top, R^3) = c_top R^2 is the Montgomery form
// of c_top R, MontMul(c_j, R^2) that of c_j, and MontMul(x, R^2) multiplies
// the value in Montgomery form by R.  Two pieces take two products.
template <int S, int TPI, int FORM>
__device__ __forceinline__ void crt_input(uint32_t (&a)[S / TPI], const uint32_t *c, bool active, int parts,
                                          const uint32_t *sR2, const uint32_t *sR3, const uint32_t (&nn)[S / TPI],
                                          uint32_t n0, uint32_t r) {
  constexpr int L = S / TPI;
  uint32_t lo[L];
  if (active) {
    load_slice_global<L>(a, c + (parts - 1) * S, r);
    load_slice_global<L>(lo, c + (parts - 2) * S, r);
  } else {
#pragma unroll
    for (int j = 0; j < L; j++) lo[j] = a[j] = 0;
  }
  mont<S, TPI, FORM>(a, sR3, nn, n0, r);   // c_top R^2
  mont<S, TPI, FORM>(lo, sR2, nn, n0, r);  // c_next R
  mod_add<L, TPI>(a, lo, nn, r);           // (c_top R + c_next) R
  for (int piece = parts - 3; piece >= 0; piece--) {
    mont<S, TPI, FORM>(a, sR2, nn, n0, r);  // value * R, still in Montgomery form
    if (active) {
      load_slice_global<L>(lo, c + piece * S, r);
    } else {
#pragma unroll
      for (int j = 0; j < L; j++) lo[j] = 0;
    }
    mont<S, TPI, FORM>(lo, sR2, nn, n0, r);
    mod_add<L, TPI>(a, lo, nn, r);
  }
}

// Which chunks a block serves, and under which key.  Every block serves one
// key, so schedules, modulus and control flow are uniform across it.
//   Round robin (grp == nullptr): blockIdx.y is the key (full width) or
//     key * parts + i (CRT, residue mod prime r_i); instance slot g of block
//     x takes the j-th chunk of that key, j = x IPB + g, chunk t = key + j K.
//   Key groups (grp != nullptr, explicit key indices): grp holds the padded
//     segment offsets poff[0..K] followed by the slot table (see
//     launch_key_groups); key k owns slots [poff[k], poff[k+1]), a multiple
//     of the table's alignment long, each holding a chunk index or
//     kNoChunk.  Block x takes slots [x IPB, (x + 1) IPB) (IPB divides the
//     alignment, so one key's), its key is found by binary search over
//     poff, and blockIdx.y is the prime.
struct BlockChunks {
  uint32_t key;
  long long first_slot;  // round robin: the block's first chunk; groups: its first slot
  bool any;              // the block has at least one chunk
};
__device__ __forceinline__ BlockChunks block_chunks(const uint32_t *__restrict__ grp, uint32_t K, long long n,
                                                    int ipb, uint32_t grid_key) {
  BlockChunks b;
  if (!grp) {
    b.key = grid_key;
    b.first_slot = grid_key + (long long)blockIdx.x * ipb * K;
    b.any = b.first_slot < n;
    return b;
  }
  const uint32_t s0 = blockIdx.x * (uint32_t)ipb;
  b.first_slot = s0;
  b.any = s0 < __ldg(grp + K);
  uint32_t lo = 0, hi = K;  // poff[lo] <= s0 < poff[hi]
  while (b.any && hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    if (__ldg(grp + mid) <= s0) lo = mid; else hi = mid;
  }
  b.key = lo;
  return b;
}
// Chunk of instance slot g (negative: none).
__device__ __forceinline__ long long slot_chunk(const uint32_t *__restrict__ grp, uint32_t K, long long n,
                                                const BlockChunks &b, uint32_t g) {
  if (!grp) {
    const long long t = b.first_slot + (long long)g * K;
    return t < n ? t : -1;
  }
  const uint32_t c = __ldg(grp + K + 1 + b.first_slot + g);
  return c == kNoChunk ? -1 : (long long)c;
}

//
// FULL: out[t] = in[t]^E mod N_key, E = e (sel != 0) or d, S = nbits / 32.
// CRT:  out[t][i] = in[t]^E mod r_i over S = nbits / (32 parts) limbs, with
//       E = d mod (r_i - 1) (sel == 0), or r_i - 2 (sel != 0: inverses mod
//       r_i by Fermat's little theorem); the input is reduced by crt_input.
//       The recombination kernel combines the residues afterwards.
// NT threads per block (128, or 64 where smaller blocks fit more
// instances in an SM's shared memory).  TABLE (kTableFull or kTableSmall)
// sizes the odd-power tables in shared memory and selects the key's
// schedules built for it.  MINB: the minimum resident blocks per SM declared
// to ptxas (0: none); 1 lets it use more registers, which pays for one
// geometry (see the CRT instantiations).  GRP = false: round robin only.
// GRP = true: a key group table (grp, explicit key indices) when grp is
// given, round robin when it is null.  Two instantiations because the table
// lookup in the prologue, though outside the exponentiation, changes how
// ptxas compiles the whole kernel: 38 instead of 32 registers at 64 limbs
// and 32 lanes, round-robin launches up to 18% slower at 100 KB, and a few
// column-form geometries 1-2% faster (measured); each geometry names the
// instantiation that serves its round-robin launches (make_entry).
template <int S, int TPI, bool CRT, int FORM, int NT = kThreads, int TABLE = kTableFull, int MINB = 0,
          bool GRP = false>
__global__ void __launch_bounds__(NT, MINB) k_modexp(const KeyDev *__restrict__ keys, uint32_t K,
                                               const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                                               long long n, int sel, int parts, const uint32_t *__restrict__ grp) {
  constexpr int L = S / TPI;
  constexpr int IPB = NT / TPI;
  constexpr int ROW = Layout<S>::kRow;
  constexpr int ROWS = table_rows(TABLE);
  constexpr int INST = Layout<S>::inst(ROWS);
  const int W = CRT ? parts * S : S;  // limbs per chunk in memory
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t *sR2 = smem, *sOne = smem + ROW, *sR3 = smem + 2 * ROW;
  const uint32_t r = threadIdx.x % TPI, g = threadIdx.x / TPI;
  uint32_t *tbl = smem + Layout<S>::kConstRows * ROW + g * INST;
  uint32_t *ybuf = tbl + ROWS * ROW;

  uint32_t key, prime;
  long long first = 0;  // round robin: the block's first chunk
  BlockChunks bc{};     // key groups: the block's key and first slot
  if constexpr (GRP) {
    prime = CRT ? (grp ? blockIdx.y : blockIdx.y % (uint32_t)parts) : 0;
    bc = block_chunks(grp, K, n, IPB, CRT ? blockIdx.y / (uint32_t)parts : blockIdx.y);
    if (!bc.any) return;  // block-uniform: no instance of this block has a chunk
    key = bc.key;
  } else {
    key = CRT ? blockIdx.y / (uint32_t)parts : blockIdx.y;
    prime = CRT ? blockIdx.y % (uint32_t)parts : 0;
    first = key + (long long)blockIdx.x * IPB * K;
    if (first >= n) return;  // block-uniform: no instance of this block has a chunk
  }
  const KeyDev &kd = keys[key];
  const uint32_t *M = CRT ? kd.P[prime] : kd.N;
  const uint32_t *R2 = CRT ? kd.R2h[prime] : kd.R2;
  const uint32_t *sched = CRT ? (sel ? kd.sched_hinv[TABLE][prime] : kd.sched_h[TABLE][prime])
                              : (sel ? kd.sched_e[TABLE] : kd.sched_d[TABLE]);
  const uint32_t nsteps = CRT ? (sel ? kd.nsteps_hinv[TABLE][prime] : kd.nsteps_h[TABLE][prime])
                              : (sel ? kd.nsteps_e[TABLE] : kd.nsteps_d[TABLE]);
  const uint32_t maxidx = CRT ? (sel ? kd.maxidx_hinv[TABLE][prime] : kd.maxidx_h[TABLE][prime])
                              : (sel ? kd.maxidx_e[TABLE] : kd.maxidx_d[TABLE]);
  const uint32_t n0 = CRT ? kd.n0h[prime] : kd.n0;

  for (int i = threadIdx.x; i < S; i += NT) {
    sR2[i] = __ldg(R2 + i);
    sOne[i] = (i == 0);
    if (CRT) sR3[i] = __ldg(kd.R3h[prime] + i);
  }
  __syncthreads();
  // After the barrier the warps are independent: a warp whose instances all
  // lie past the last chunk of the key leaves (chunks and slots of a key are
  // in order, padding last, so its first instance decides).
  long long t;
  bool active;
  if constexpr (GRP) {
    if (slot_chunk(grp, K, n, bc, (threadIdx.x / 32) * (32 / TPI)) < 0) return;
    t = slot_chunk(grp, K, n, bc, g);
    active = t >= 0;
  } else {
    if (first + (long long)((threadIdx.x / 32) * (32 / TPI)) * K >= n) return;
    t = first + (long long)g * K;
    active = t < n;
  }
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
    crt_input<S, TPI, FORM>(a, in + t * W, active, parts, sR2, sR3, nn, n0, r);
  }
  exp_window<S, TPI, FORM>(a, tbl, ybuf, sched, nsteps, maxidx, nn, n0, r);
  mont<S, TPI, FORM>(a, sOne, nn, n0, r);  // leave the Montgomery domain
  if (active) {
    uint32_t *o = out + t * W + (CRT ? prime * S : 0) + r * L;
    if constexpr (L % 4 == 0) {
#pragma unroll
      for (int j = 0; j < L; j += 4) *reinterpret_cast<uint4 *>(o + j) = make_uint4(a[j], a[j + 1], a[j + 2], a[j + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < L; j++) o[j] = a[j];
    }
  }
}

}  // namespace dev
}  // namespace pmk
