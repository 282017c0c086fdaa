// Warp-cooperative Montgomery exponentiation for sm_103a.
//
// One exponentiation ("instance") is held by TPI consecutive lanes of a warp;
// lane r keeps limbs [r L, r L + L) of every S-limb value in registers
// (L = S / TPI).  The multiplication is Algorithm 3 (Montgomery) in its
// word-serial CIOS form (Koc, Acar, Kaliski 1996) with r = 2^32 per row and
// R = 2^(32 S) overall:
//     for i in 0..S-1:  T += a * y_i;  q = T_0 * n0 mod 2^32;  T += q N;  T /= 2^32
// followed by one conditional subtraction, so every product is canonical
// (< N).  Exponentiation is Algorithm 2's square-and-multiply generalised to a
// left-to-right sliding window of odd powers (schedules built on the host).
//
// Cost model on this GPU (measured with row-shaped loops, one multiplier per
// row and the multiplicands in registers): mad.lo issues at up to 64
// lanes/clk/SM but the high half of a 32x32 product at only about 22, and a
// wide multiply (both halves, with or without a 64-bit addend) at 16-24
// depending on the warps per SM.  The high half is therefore the cost of a
// MAC whatever form it takes.  Integer adds issue on the ALU pipe, in
// parallel.  So each row forms its L products with wide multiplies and folds
// them in with two add-with-carry chains (low halves at word j, high halves
// at word j + 1).
// Lane-to-lane carries are deferred: a lane keeps a small pending word above
// its L limbs, which the per-row shift moves into its own top limb; after the
// last row a ballot carry-lookahead resolves them in O(1) warp operations.
#pragma once

#include <cstdint>

#include "pmk_internal.h"

namespace pmk {
namespace dev {

constexpr int kThreads = 128;   // threads per block (4 warps)
constexpr int kTableMax = 1 << (kWindowFull - 1);  // odd powers x^1 .. x^(2 kTableMax - 1)
// Rows of the odd-power table of each size (kTableFull, kTableSmall).
__host__ __device__ constexpr int table_rows(int table) { return table == kTableSmall ? kTableMax / 2 : kTableMax; }
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void add_cc(uint32_t &r, uint32_t a, uint32_t b) {
  asm volatile("add.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
}
__device__ __forceinline__ void addc_cc(uint32_t &r, uint32_t a, uint32_t b) {
  asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
}
__device__ __forceinline__ void addc(uint32_t &r, uint32_t a, uint32_t b) {
  asm volatile("addc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
}
__device__ __forceinline__ void sub_cc(uint32_t &r, uint32_t a, uint32_t b) {
  asm volatile("sub.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
}
__device__ __forceinline__ void subc_cc(uint32_t &r, uint32_t a, uint32_t b) {
  asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
}
__device__ __forceinline__ void subc(uint32_t &r, uint32_t a, uint32_t b) {
  asm volatile("subc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
}

// Words of shared memory per stored S-limb value: S + 4 keeps 16-byte rows.
template <int S>
struct Layout {
  static constexpr int kRow = S + 4;
  // Per-instance block (a table of `rows` rows + one operand buffer), padded
  // to 4 mod 32 words so the 32/TPI instances of a warp read distinct
  // 16-byte bank groups.
  static __host__ __device__ constexpr int inst(int rows) {
    return (rows + 1) * kRow + ((4 - ((rows + 1) * kRow) % 32) + 32) % 32;
  }
  static constexpr int kInst = inst(kTableMax);
  static constexpr int kConstRows = 3;  // R^2, one, R^3
};

// Row forms: how one row t += a * y turns into instructions.
//   kWide: L wide multiplies (64-bit products), low and high halves folded in
//          by two add-with-carry chains on the integer ALU pipe;
//   kMadc: mad.lo/mad.hi with carry in and out, so the multiply unit also
//          does the additions (nothing on the ALU pipe but the chain ends).
// A Montgomery row pair (a * y_i, then q * N) may use a different form for
// each half, to balance the multiply and ALU pipes.
enum RowForm : int { kWide = 0, kMadc = 1 };
#ifndef PMK_ROW_FORM
#define PMK_ROW_FORM 0
#endif
constexpr int kFormA = (PMK_ROW_FORM == 1 || PMK_ROW_FORM == 2) ? kMadc : kWide;  // a * y_i
constexpr int kFormN = (PMK_ROW_FORM == 1 || PMK_ROW_FORM == 3) ? kMadc : kWide;  // q * N

__device__ __forceinline__ void madlo_cc(uint32_t &t, uint32_t a, uint32_t y) {
  asm volatile("mad.lo.cc.u32 %0, %1, %2, %0;" : "+r"(t) : "r"(a), "r"(y));
}
__device__ __forceinline__ void madclo_cc(uint32_t &t, uint32_t a, uint32_t y) {
  asm volatile("madc.lo.cc.u32 %0, %1, %2, %0;" : "+r"(t) : "r"(a), "r"(y));
}
__device__ __forceinline__ void madhi_cc(uint32_t &t, uint32_t a, uint32_t y) {
  asm volatile("mad.hi.cc.u32 %0, %1, %2, %0;" : "+r"(t) : "r"(a), "r"(y));
}
__device__ __forceinline__ void madchi_cc(uint32_t &t, uint32_t a, uint32_t y) {
  asm volatile("madc.hi.cc.u32 %0, %1, %2, %0;" : "+r"(t) : "r"(a), "r"(y));
}

// (t, c0, c1) += a * y, where t is this lane's L limbs and (c0, c1) the
// pending words above them.
template <int L, int FORM>
__device__ __forceinline__ void row_mac(uint32_t (&t)[L], uint32_t &c0, uint32_t &c1, const uint32_t (&a)[L],
                                        uint32_t y) {
  if constexpr (FORM == kMadc) {
    madlo_cc(t[0], a[0], y);
#pragma unroll
    for (int j = 1; j < L; j++) madclo_cc(t[j], a[j], y);
    addc_cc(c0, c0, 0u);
    addc(c1, c1, 0u);
    if constexpr (L > 1) {
      madhi_cc(t[1], a[0], y);
#pragma unroll
      for (int j = 1; j < L - 1; j++) madchi_cc(t[j + 1], a[j], y);
      madchi_cc(c0, a[L - 1], y);
    } else {
      madhi_cc(c0, a[0], y);
    }
    addc(c1, c1, 0u);
    return;
  }
  uint32_t lo[L], hi[L];
#pragma unroll
  for (int j = 0; j < L; j++) {
    const uint64_t p = (uint64_t)a[j] * y;
    lo[j] = (uint32_t)p;
    hi[j] = (uint32_t)(p >> 32);
  }
  add_cc(t[0], t[0], lo[0]);
#pragma unroll
  for (int j = 1; j < L; j++) addc_cc(t[j], t[j], lo[j]);
  addc_cc(c0, c0, 0u);
  addc(c1, c1, 0u);
  if constexpr (L > 1) {
    add_cc(t[1], t[1], hi[0]);
#pragma unroll
    for (int j = 1; j < L - 1; j++) addc_cc(t[j + 1], t[j + 1], hi[j]);
    addc_cc(c0, c0, hi[L - 1]);
  } else {
    add_cc(c0, c0, hi[0]);
  }
  addc(c1, c1, 0u);
}

// Carry-lookahead over the lanes of every TPI-lane group of the warp.
// gen: this lane's word-block overflowed into the next lane; prop: this
// lane's block is all ones (all zeros for borrows) and passes a carry on.
// Returns the carry (0/1) entering this lane.  Top lanes of a group neither
// generate nor propagate into the next group.
__device__ __forceinline__ uint32_t lookahead(bool gen, bool prop, bool top) {
  const uint32_t G = __ballot_sync(kFull, gen && !top);
  const uint32_t P = __ballot_sync(kFull, prop && !top);
  const uint32_t cin = ((G | P) + G) ^ P;  // carry into each bit of (G|P) + G
  return (cin >> (threadIdx.x & 31)) & 1u;
}

// Resolve the pending word c0 (lane r's belongs at lane r+1's limb 0; the top
// lane's is the value's top word) and reduce the value once by N, leaving the
// canonical result (< N) in t.  Requires the value < 2N.
template <int L, int TPI>
__device__ __forceinline__ void finalize(uint32_t (&t)[L], uint32_t c0, const uint32_t (&nn)[L], uint32_t r) {
  const bool top = (r == TPI - 1);
  uint32_t topw = top ? c0 : 0u;
  if constexpr (TPI > 1) {
    uint32_t inc = __shfl_up_sync(kFull, c0, 1, TPI);
    if (r == 0) inc = 0;
    uint32_t g;
    add_cc(t[0], t[0], inc);
#pragma unroll
    for (int j = 1; j < L; j++) addc_cc(t[j], t[j], 0u);
    addc(g, 0u, 0u);
    uint32_t all1 = t[0];
#pragma unroll
    for (int j = 1; j < L; j++) all1 &= t[j];
    const uint32_t cin = lookahead(g != 0, all1 == 0xffffffffu, top);
    uint32_t g2;
    add_cc(t[0], t[0], cin);
#pragma unroll
    for (int j = 1; j < L; j++) addc_cc(t[j], t[j], 0u);
    addc(g2, 0u, 0u);
    if (top) topw += g + g2;
  }
  uint32_t d[L], b;
  sub_cc(d[0], t[0], nn[0]);
#pragma unroll
  for (int j = 1; j < L; j++) subc_cc(d[j], t[j], nn[j]);
  subc(b, 0u, 0u);
  b &= 1u;
  if constexpr (TPI > 1) {
    uint32_t any = d[0];
#pragma unroll
    for (int j = 1; j < L; j++) any |= d[j];
    const uint32_t bin = lookahead(b != 0, any == 0, top);
    uint32_t b2;
    sub_cc(d[0], d[0], bin);
#pragma unroll
    for (int j = 1; j < L; j++) subc_cc(d[j], d[j], 0u);
    subc(b2, 0u, 0u);
    b |= b2 & 1u;
  }
  // value - N = (topw - b) 2^(32 S) + d: keep d iff topw >= b (decided by the top lane)
  uint32_t ge = (topw >= b) ? 1u : 0u;
  if constexpr (TPI > 1) ge = __shfl_sync(kFull, ge, TPI - 1, TPI);
  if (ge) {
#pragma unroll
    for (int j = 0; j < L; j++) t[j] = d[j];
  }
}

// Rows of a product processed per unrolled group (y limbs fetched as 16- or
// 8-byte broadcasts).  In the carry-chain form a group of L rows (L = limbs
// per lane, 6 to 16) brings the per-row shift of the lane's words back to
// the starting registers, so no register moves remain: measured 3-18%
// faster than groups of 4 at 6, 8, 12 and 16 limbs per lane.  The column
// form measured no gain and keeps groups of 4.
template <int S, int L, bool kChainForm>
__host__ __device__ constexpr int row_group() {
  return (kChainForm && L >= 6 && L <= 16 && L % 2 == 0 && S % L == 0) ? L : (S % 4 == 0) ? 4 : 2;
}

template <int K>
__device__ __forceinline__ void load_y(uint32_t (&yv)[K], const uint32_t *ys) {
  if constexpr (K % 4 == 0) {
#pragma unroll
    for (int q = 0; q < K; q += 4) {
      const uint4 v = *reinterpret_cast<const uint4 *>(ys + q);
      yv[q] = v.x; yv[q + 1] = v.y; yv[q + 2] = v.z; yv[q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < K; q += 2) {
      const uint2 v = *reinterpret_cast<const uint2 *>(ys + q);
      yv[q] = v.x; yv[q + 1] = v.y;
    }
  }
}

// a <- MontMul(a, y) = a y R^-1 mod N.  a: this lane's limbs (any value < R);
// ys: y's S limbs in shared memory (y < N), read as 16-byte broadcasts.
template <int S, int TPI>
__device__ __forceinline__ void mont_mul(uint32_t (&a)[S / TPI], const uint32_t *ys, const uint32_t (&nn)[S / TPI],
                                         uint32_t n0, uint32_t r) {
  constexpr int L = S / TPI;
  constexpr int kStep = row_group<S, L, true>();
  uint32_t t[L];
#pragma unroll
  for (int j = 0; j < L; j++) t[j] = 0;
  uint32_t c0 = 0, c1 = 0;
#pragma unroll 1
  for (int i0 = 0; i0 < S; i0 += kStep) {
    uint32_t yv[kStep];
    load_y<kStep>(yv, ys + i0);
#pragma unroll
    for (int u = 0; u < kStep; u++) {
      row_mac<L, kFormA>(t, c0, c1, a, yv[u]);
      uint32_t q = t[0] * n0;
      if constexpr (TPI > 1) q = __shfl_sync(kFull, q, 0, TPI);
      row_mac<L, kFormN>(t, c0, c1, nn, q);
      // T /= 2^32: limb 0 of lane 0 is now zero; every lane takes the next
      // lane's limb 0 as its new top limb and folds its pending word into it.
      uint32_t in = 0;
      if constexpr (TPI > 1) {
        in = __shfl_down_sync(kFull, t[0], 1, TPI);
        if (r == TPI - 1) in = 0;
      }
#pragma unroll
      for (int j = 0; j < L - 1; j++) t[j] = t[j + 1];
      add_cc(t[L - 1], in, c0);
      addc(c0, c1, 0u);
      c1 = 0;
    }
  }
  finalize<L, TPI>(t, c0, nn, r);
#pragma unroll
  for (int j = 0; j < L; j++) a[j] = t[j];
}

// a <- MontMul(a, y), column form.  Each lane keeps one 64-bit accumulator
// per limb position ("column"): the low half of a product a_j * y_i goes to
// column j and its high half to column j + 1, so a row is L independent
// column updates instead of one add-with-carry chain through the lane.
// Columns absorb at most four 32-bit terms per row and live at most S + L
// rows, so they stay below 2^42.  The row shift moves a whole column (two
// shuffles); column carries are propagated once, before finalize.
template <int S, int TPI>
__device__ __forceinline__ void mont_mul_cols(uint32_t (&a)[S / TPI], const uint32_t *ys, const uint32_t (&nn)[S / TPI],
                                              uint32_t n0, uint32_t r) {
  constexpr int L = S / TPI;
  constexpr int kStep = row_group<S, L, false>();
  uint64_t acc[L];
#pragma unroll
  for (int j = 0; j < L; j++) acc[j] = 0;
#pragma unroll 1
  for (int i0 = 0; i0 < S; i0 += kStep) {
    uint32_t yv[kStep];
    load_y<kStep>(yv, ys + i0);
#pragma unroll
    for (int u = 0; u < kStep; u++) {
      uint32_t hprev = 0;
#pragma unroll
      for (int j = 0; j < L; j++) {
        const uint64_t p = (uint64_t)a[j] * yv[u];
        acc[j] += (uint64_t)(uint32_t)p + hprev;
        hprev = (uint32_t)(p >> 32);
      }
      uint64_t top = hprev;  // column L: the next lane's column 0 before the shift
      uint32_t q = (uint32_t)acc[0] * n0;
      if constexpr (TPI > 1) q = __shfl_sync(kFull, q, 0, TPI);
      hprev = 0;
#pragma unroll
      for (int j = 0; j < L; j++) {
        const uint64_t p = (uint64_t)nn[j] * q;
        acc[j] += (uint64_t)(uint32_t)p + hprev;
        hprev = (uint32_t)(p >> 32);
      }
      top += hprev;
      // T /= 2^32: column 0 of lane 0 is now zero mod 2^32 and its high part
      // carries into column 1; every other lane's column 0 moves down to the
      // previous lane's top column.
      uint64_t in = 0;
      if constexpr (TPI > 1) {
        const uint32_t lo = __shfl_down_sync(kFull, (uint32_t)acc[0], 1, TPI);
        const uint32_t hi = __shfl_down_sync(kFull, (uint32_t)(acc[0] >> 32), 1, TPI);
        if (r != TPI - 1) in = ((uint64_t)hi << 32) | lo;
      }
      const uint64_t carry0 = (r == 0) ? (acc[0] >> 32) : 0;
#pragma unroll
      for (int j = 0; j < L - 1; j++) acc[j] = acc[j + 1];
      acc[L - 1] = in + top;
      acc[0] += carry0;
    }
  }
  uint32_t t[L];
  uint64_t c = 0;
#pragma unroll
  for (int j = 0; j < L; j++) {
    const uint64_t v = acc[j] + c;
    t[j] = (uint32_t)v;
    c = v >> 32;
  }
  finalize<L, TPI>(t, (uint32_t)c, nn, r);
#pragma unroll
  for (int j = 0; j < L; j++) a[j] = t[j];
}

// Montgomery product forms: kChain = mont_mul (one add-with-carry chain per
// lane and row), kCols = mont_mul_cols (independent 64-bit columns).  Which is
// faster depends on limbs per lane and on how many warps a batch provides, so
// each compiled geometry names its form.
enum MontForm : int { kChain = 0, kCols = 1 };

template <int S, int TPI, int FORM>
__device__ __forceinline__ void mont(uint32_t (&a)[S / TPI], const uint32_t *ys, const uint32_t (&nn)[S / TPI],
                                     uint32_t n0, uint32_t r) {
  if constexpr (FORM == kCols) {
    mont_mul_cols<S, TPI>(a, ys, nn, n0, r);
  } else {
    mont_mul<S, TPI>(a, ys, nn, n0, r);
  }
}

// a <- (a + b) mod N for a, b < N (distributed add, lookahead, one reduction).
template <int L, int TPI>
__device__ __forceinline__ void mod_add(uint32_t (&a)[L], const uint32_t (&b)[L], const uint32_t (&nn)[L], uint32_t r) {
  uint32_t c;
  add_cc(a[0], a[0], b[0]);
#pragma unroll
  for (int j = 1; j < L; j++) addc_cc(a[j], a[j], b[j]);
  addc(c, 0u, 0u);
  // c is this lane's carry into the next lane: reuse finalize, whose first
  // step moves a lane's pending word into the next lane's limb 0.
  finalize<L, TPI>(a, c, nn, r);
}

// Store / load this lane's L limbs of a value at row + r L.
template <int L>
__device__ __forceinline__ void store_slice(uint32_t *row, const uint32_t (&a)[L], uint32_t r) {
  uint32_t *p = row + r * L;
  if constexpr (L % 4 == 0) {
#pragma unroll
    for (int j = 0; j < L; j += 4) *reinterpret_cast<uint4 *>(p + j) = make_uint4(a[j], a[j + 1], a[j + 2], a[j + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < L; j++) p[j] = a[j];
  }
}
template <int L>
__device__ __forceinline__ void load_slice(uint32_t (&a)[L], const uint32_t *row, uint32_t r) {
  const uint32_t *p = row + r * L;
  if constexpr (L % 4 == 0) {
#pragma unroll
    for (int j = 0; j < L; j += 4) {
      const uint4 v = *reinterpret_cast<const uint4 *>(p + j);
      a[j] = v.x; a[j + 1] = v.y; a[j + 2] = v.z; a[j + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < L; j++) a[j] = p[j];
  }
}
template <int L>
__device__ __forceinline__ void load_slice_global(uint32_t (&a)[L], const uint32_t *__restrict__ row, uint32_t r) {
  const uint32_t *p = row + r * L;
  if constexpr (L % 4 == 0) {
#pragma unroll
    for (int j = 0; j < L; j += 4) {
      const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p + j));
      a[j] = v.x; a[j + 1] = v.y; a[j + 2] = v.z; a[j + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < L; j++) a[j] = __ldg(p + j);
  }
}

// Table of odd powers and the exponent walk.  On entry a = x in Montgomery
// form; on exit a = x^E in Montgomery form.  tbl: the instance's odd-power
// table (at least maxidx + 1 rows: the table size the schedule was built
// for), ybuf: one row of this instance.  sched: steps of make_schedule()
// (block-uniform).
template <int S, int TPI, int FORM>
__device__ __forceinline__ void exp_window(uint32_t (&a)[S / TPI], uint32_t *tbl, uint32_t *ybuf,
                                           const uint32_t *__restrict__ sched, uint32_t nsteps, uint32_t maxidx,
                                           const uint32_t (&nn)[S / TPI], uint32_t n0, uint32_t r) {
  constexpr int L = S / TPI;
  constexpr int ROW = Layout<S>::kRow;
  store_slice<L>(tbl, a, r);  // T[0] = x
  if (maxidx > 0) {
    store_slice<L>(ybuf, a, r);
    __syncwarp();
    mont<S, TPI, FORM>(a, ybuf, nn, n0, r);  // x^2
    __syncwarp();
    store_slice<L>(ybuf, a, r);
    load_slice<L>(a, tbl, r);
    __syncwarp();
#pragma unroll 1
    for (uint32_t k = 1; k <= maxidx; k++) {  // T[k] = T[k-1] x^2 = x^(2k+1)
      mont<S, TPI, FORM>(a, ybuf, nn, n0, r);
      store_slice<L>(tbl + k * ROW, a, r);
    }
    __syncwarp();
  }
  load_slice<L>(a, tbl + __ldg(sched) * ROW, r);
#pragma unroll 1
  for (uint32_t si = 1; si < nsteps; si++) {
    const uint32_t step = __ldg(sched + si);
    const uint32_t nsq = step >> 8, idx = step & 0xffu;
#pragma unroll 1
    for (uint32_t k = 0; k < nsq; k++) {
      __syncwarp();
      store_slice<L>(ybuf, a, r);
      __syncwarp();
      mont<S, TPI, FORM>(a, ybuf, nn, n0, r);
    }
    if (idx != 0xffu) mont<S, TPI, FORM>(a, tbl + idx * ROW, nn, n0, r);
  }
}

}  // namespace dev
}  // namespace pmk
