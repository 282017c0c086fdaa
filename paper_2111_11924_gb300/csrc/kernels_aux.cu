// Split / join (HBM-bound byte <-> limb repacking), the input range check, the
// thread-per-chunk baseline, and the launchers of the exponentiation,
// modular-multiplication and CRT-recombination kernels.
#include <algorithm>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "modexp_kernels.cuh"

namespace pmk {
namespace {

constexpr int kAuxThreads = 256;

// Division of numerators below 2^31 by a run-time constant d (Granlund and
// Montgomery, PLDI 1994): q = floor(x M / 2^(31 + s)) with s = ceil(log2 d)
// and M = ceil(2^(31 + s) / d) < 2^32.  Exact: writing M d = 2^(31+s) + e
// with 0 <= e < d, the excess x e / (d 2^(31+s)) is below 2^-s <= 1/d.
struct DivMagic {
  uint32_t M;
  int sh;  // s - 1; -1 for d = 1
};

DivMagic div_magic(uint32_t d) {
  if (d <= 1) return DivMagic{1u, -1};
  int s = 0;
  while ((1ull << s) < d) s++;
  const unsigned long long M = ((1ull << (31 + s)) + d - 1) / d;
  return DivMagic{(uint32_t)M, s - 1};
}

// x / d: the magic multiply for 32-bit indices (x < 2^31), plain division otherwise.
template <typename I>
__device__ __forceinline__ I quot(I x, uint32_t d, DivMagic m) {
  if constexpr (sizeof(I) == 4) {
    return m.sh < 0 ? x : (__umulhi(x, m.M) >> m.sh);
  } else {
    return x / d;
  }
}

// The 16 bytes starting at byte `off` (0..16) of the 32 bytes (lo, hi).
__device__ __forceinline__ uint4 bytes_at(const uint4 lo, const uint4 hi, uint32_t off) {
  const uint32_t x[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
  const uint32_t sh = (off & 3u) * 8u;
  uint32_t w[4];
  switch (off >> 2) {
#define PMK_CASE(WO)                                                                 \
  case WO:                                                                           \
    for (int k = 0; k < 4; k++) w[k] = __funnelshift_r(x[k + WO], x[k + WO + 1], sh); \
    break;
    PMK_CASE(0)
    PMK_CASE(1)
    PMK_CASE(2)
    case 3:
      for (int k = 0; k < 4; k++) w[k] = __funnelshift_r(x[k + 3], x[k + 4], sh);
      break;
    default:
      return hi;
#undef PMK_CASE
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Word k of the mask of bytes [0, n) of a 16-byte vector.
__device__ __forceinline__ uint32_t keep_mask(int n, int k) {
  const int c = n - 4 * k;
  return c >= 4 ? 0xffffffffu : c <= 0 ? 0u : (0xffffffffu >> (32 - 8 * c));
}

// A chunk holds nbits/8 = P + 1 bytes, so the limb buffer is the message
// with one zero byte (the "pad") after every P message bytes: chunk byte j
// of chunk t is message byte t P + j for j < P, and zero for j = P.

// Split (Section 3.1): word j of chunk t holds message bytes t P + 4j .. +3
// (little-endian), zero past the chunk payload P or the message end L.
// One thread per 16 output bytes: limb vector v of the buffer starts at
// message byte 16 v - t (t = v / (S/4), its chunk), so it is the 16-byte
// window there -- two aligned 16-byte loads and a byte shift -- with the pad
// byte cleared in a chunk's last vector.  The message tail, and a message
// that does not start on a 16-byte boundary, go byte by byte.
template <typename I>
__global__ void __launch_bounds__(kAuxThreads) k_split(const uint8_t *__restrict__ msg, I L, int P, int S,
                                                       uint4 *__restrict__ out, I nvec, int msg_aligned,
                                                       DivMagic mvpc) {
  const I vpc = (I)(S / 4);  // vectors per chunk
  const uint4 *msg16 = reinterpret_cast<const uint4 *>(msg);
  (void)P;
  for (I v = (I)blockIdx.x * kAuxThreads + threadIdx.x; v < nvec; v += (I)gridDim.x * kAuxThreads) {
    const I t = quot<I>(v, (uint32_t)vpc, mvpc);
    const I m0 = v * 16 - t;
    uint4 r = make_uint4(0, 0, 0, 0);
    if (m0 < L) {
      const I a = m0 >> 4;
      if (msg_aligned && (a + 2) * 16 <= L) {
        r = bytes_at(__ldg(msg16 + a), __ldg(msg16 + a + 1), (uint32_t)(m0 & 15));
      } else {
        uint32_t w[4] = {0, 0, 0, 0};
        for (int i = 0; i < 16 && m0 + i < L; i++) w[i >> 2] |= (uint32_t)__ldg(msg + m0 + i) << (8 * (i & 3));
        r = make_uint4(w[0], w[1], w[2], w[3]);
      }
      if (v - t * vpc == vpc - 1) r.w &= 0x00ffffffu;  // chunk byte P: the pad
    }
    out[v] = r;
  }
}

// Join: byte b of the message is byte (b mod P) of chunk b / P, i.e. byte
// b + b / P of the limb buffer.  One thread per 16 message bytes: the 17
// buffer bytes from b0 + t (t = b0 / P) hold them, with the pad inside when
// the vector crosses into chunk t + 1 after n1 = P - (b0 mod P) < 16 bytes;
// then bytes [0, n1) come from the window at b0 + t and the rest from the
// window one byte later.  One 16-byte store writes the vector; the message
// tail (or an unaligned output) is written byte by byte.
template <typename I>
__global__ void __launch_bounds__(kAuxThreads) k_join(const uint32_t *__restrict__ chunks, int P, int S,
                                                      uint8_t *__restrict__ msg, I L, int out_aligned,
                                                      DivMagic mP, I nbuf16) {
  const I nvec = (L + 15) / 16;
  const uint4 *c16 = reinterpret_cast<const uint4 *>(chunks);
  (void)S;
  for (I u = (I)blockIdx.x * kAuxThreads + threadIdx.x; u < nvec; u += (I)gridDim.x * kAuxThreads) {
    const I b0 = u * 16;
    const I t = quot<I>(b0, (uint32_t)P, mP);
    const int n1 = P - (int)(b0 - t * (I)P);  // bytes left in chunk t (>= 1)
    const I src0 = b0 + t;
    const I a = src0 >> 4;
    const uint32_t off = (uint32_t)(src0 & 15);
    const uint4 lo = __ldg(c16 + a);
    const uint4 hi = (a + 1 < nbuf16) ? __ldg(c16 + a + 1) : make_uint4(0, 0, 0, 0);
    uint4 r = bytes_at(lo, hi, off);
    if (n1 < 16) {  // skip the pad byte at position n1
      const uint4 r1 = bytes_at(lo, hi, off + 1);
      const uint32_t m0 = keep_mask(n1, 0), m1 = keep_mask(n1, 1), m2 = keep_mask(n1, 2), m3 = keep_mask(n1, 3);
      r = make_uint4((r.x & m0) | (r1.x & ~m0), (r.y & m1) | (r1.y & ~m1), (r.z & m2) | (r1.z & ~m2),
                     (r.w & m3) | (r1.w & ~m3));
    }
    if (out_aligned && b0 + 16 <= L) {
      reinterpret_cast<uint4 *>(msg)[u] = r;
    } else {
      const uint32_t w[4] = {r.x, r.y, r.z, r.w};
      for (int i = 0; i < 16 && b0 + i < L; i++) msg[b0 + i] = (uint8_t)(w[i >> 2] >> (8 * (i & 3)));
    }
  }
}

// Flags chunks whose value is >= the modulus of their key (t mod K, or
// key_idx[t]); a key index >= K flags kStatusKeyIndex instead.
__global__ void __launch_bounds__(kAuxThreads) k_range(const KeyDev *__restrict__ keys, uint32_t K, int S,
                                                       const uint32_t *__restrict__ in, long long n,
                                                       uint32_t *__restrict__ status,
                                                       const uint32_t *__restrict__ key_idx) {
  const long long t = (long long)blockIdx.x * kAuxThreads + threadIdx.x;
  if (t >= n) return;
  const uint32_t *x = in + t * S;
  const uint32_t k = key_idx ? __ldg(key_idx + t) : (uint32_t)(t % K);
  if (k >= K) {
    report(status, kStatusKeyIndex, t);
    return;
  }
  const uint32_t *N = keys[k].N;
  int ge = 1;  // x == N counts as out of range
  for (int i = S - 1; i >= 0; i--) {
    const uint32_t xi = __ldg(x + i), ni = __ldg(N + i);
    if (xi != ni) {
      ge = xi > ni;
      break;
    }
  }
  if (ge) report(status, kStatusRange, t);
}

// Key groups for explicit key indices, in three passes.
//   count:   histogram of the indices (a shared-memory histogram per block,
//            added into count[0..K) once per bin);
//   offsets: poff[k] = sum over j < k of count[j] rounded up to the table's
//            alignment, poff[K] the total (one block; also cursor[k] = poff[k]);
//   scatter: slot[cursor[k]++] = t for every chunk t of key k.  The lanes of
//            a warp with equal keys take consecutive slots with one atomic.
// The slot table starts filled with kNoChunk (the padding).  Slot order
// within a key follows the atomics, so it may vary from call to call; each
// chunk's result does not depend on it.
__global__ void __launch_bounds__(kAuxThreads) k_key_count(const uint32_t *__restrict__ key_idx, long long n,
                                                           uint32_t K, uint32_t *__restrict__ count,
                                                           uint32_t *__restrict__ status) {
  extern __shared__ uint32_t hist[];
  for (uint32_t k = threadIdx.x; k < K; k += kAuxThreads) hist[k] = 0;
  __syncthreads();
  for (long long t = (long long)blockIdx.x * kAuxThreads + threadIdx.x; t < n; t += (long long)gridDim.x * kAuxThreads) {
    const uint32_t k = __ldg(key_idx + t);
    if (k < K) atomicAdd(&hist[k], 1u); else report(status, kStatusKeyIndex, t);
  }
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < K; k += kAuxThreads)
    if (hist[k]) atomicAdd(count + k, hist[k]);
}

constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) k_key_offsets(const uint32_t *__restrict__ count, uint32_t K,
                                                              uint32_t align, uint32_t *__restrict__ poff,
                                                              uint32_t *__restrict__ cursor) {
  __shared__ uint32_t part[kScanThreads];
  const uint32_t per = (K + kScanThreads - 1) / kScanThreads;  // keys per thread, contiguous
  const uint32_t k0 = threadIdx.x * per, k1 = min(K, k0 + per);
  uint32_t sum = 0;
  for (uint32_t k = k0; k < k1; k++) sum += (count[k] + align - 1) / align * align;
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int d = 1; d < kScanThreads; d <<= 1) {  // inclusive scan (Hillis-Steele)
    const uint32_t v = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t off = part[threadIdx.x] - sum;  // exclusive prefix of this thread's keys
  for (uint32_t k = k0; k < k1; k++) {
    poff[k] = off;
    cursor[k] = off;
    off += (count[k] + align - 1) / align * align;
  }
  if (threadIdx.x == kScanThreads - 1) poff[K] = part[threadIdx.x];
}

__global__ void __launch_bounds__(kAuxThreads) k_key_scatter(const uint32_t *__restrict__ key_idx, long long n,
                                                             uint32_t K, uint32_t *__restrict__ cursor,
                                                             uint32_t *__restrict__ slot) {
  const long long base = (long long)blockIdx.x * kAuxThreads;
  for (long long t0 = base; t0 < n; t0 += (long long)gridDim.x * kAuxThreads) {
    const long long t = t0 + threadIdx.x;
    const bool live = t < n;  // uniform loop bound: every lane of the warp reaches the match below
    const uint32_t k = live ? __ldg(key_idx + t) : kNoChunk;
    const uint32_t peers = __match_any_sync(dev::kFull, k);
    if (!live || k >= K) continue;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    uint32_t pos = 0;
    if (lane == leader) pos = atomicAdd(cursor + k, (uint32_t)__popc(peers));
    pos = __shfl_sync(peers, pos, leader);
    slot[pos + rank] = (uint32_t)t;
  }
}

// The plain GPU formulation, kept as a measured baseline: one thread per
// chunk, its S-limb values in local memory, single-thread CIOS Montgomery
// products and Algorithm 2's binary exponentiation (right-to-left, as printed).
// out[t] = in[t]^E mod N_{t mod K}, E = e (enc) or d.
template <int S>
__global__ void __launch_bounds__(128) k_modexp_naive(const KeyDev *__restrict__ keys, uint32_t K,
                                                      const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                                                      long long n, int enc) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const KeyDev &kd = keys[t % K];
  const uint32_t *N = kd.N, n0 = kd.n0;
  uint32_t x[S], y[S], acc[S + 2];
  auto montmul = [&](uint32_t *a, const uint32_t *b) {  // a <- a b R^-1 mod N
    for (int i = 0; i < S + 2; i++) acc[i] = 0;
    for (int i = 0; i < S; i++) {
      uint64_t c = 0;
      for (int j = 0; j < S; j++) {
        c += (uint64_t)a[j] * b[i] + acc[j];
        acc[j] = (uint32_t)c;
        c >>= 32;
      }
      c += acc[S];
      acc[S] = (uint32_t)c;
      acc[S + 1] = (uint32_t)(c >> 32);
      const uint32_t q = acc[0] * n0;
      c = ((uint64_t)q * N[0] + acc[0]) >> 32;
      for (int j = 1; j < S; j++) {
        c += (uint64_t)q * N[j] + acc[j];
        acc[j - 1] = (uint32_t)c;
        c >>= 32;
      }
      c += acc[S];
      acc[S - 1] = (uint32_t)c;
      acc[S] = acc[S + 1] + (uint32_t)(c >> 32);
    }
    uint32_t d[S], borrow = 0;
    for (int i = 0; i < S; i++) {
      const uint64_t v = (uint64_t)acc[i] - N[i] - borrow;
      d[i] = (uint32_t)v;
      borrow = (uint32_t)(v >> 63);
    }
    const bool ge = acc[S] || !borrow;
    for (int i = 0; i < S; i++) a[i] = ge ? d[i] : acc[i];
  };
  const uint32_t *E = enc ? kd.e_limbs : kd.d_limbs;  // the exponent itself, bit by bit
  const int ne = enc ? 2 : S;
  for (int i = 0; i < S; i++) x[i] = in[t * S + i];
  for (int i = 0; i < S; i++) y[i] = kd.R2[i];
  montmul(x, y);                      // x R
  for (int i = 0; i < S; i++) y[i] = (i == 0);
  montmul(y, kd.R2);                  // y = R mod N (one)
  int top = -1;
  for (int i = 32 * ne - 1; i >= 0 && top < 0; i--)
    if ((E[i / 32] >> (i % 32)) & 1) top = i;
  for (int i = 0; i < top; i++) {     // Algorithm 2: bits e_0 .. e_{l-1}
    if ((E[i / 32] >> (i % 32)) & 1) montmul(y, x);
    uint32_t xc[S];
    for (int j = 0; j < S; j++) xc[j] = x[j];
    montmul(x, xc);
  }
  montmul(y, x);                      // the top bit
  for (int i = 0; i < S; i++) x[i] = (i == 0);
  montmul(y, x);                      // leave the Montgomery domain
  for (int i = 0; i < S; i++) out[t * S + i] = y[i];
}

int grid_for(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  return (int)std::max(1LL, std::min(b, 152LL * 64));
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? PMK_OK : PMK_ECUDA; }

// Every compiled instantiation of one mode (the wide-key list is shared).
std::vector<ModexpEntry> entries(bool crt) {
  int n = 0, m = 0;
  const ModexpEntry *list = crt ? modexp_entries_crt(&n) : modexp_entries_full(&n);
  const ModexpEntry *wide = modexp_entries_wide(&m);
  std::vector<ModexpEntry> v(list, list + n);
  for (int i = 0; i < m; i++)
    if (wide[i].crt == crt) v.push_back(wide[i]);
  const ModexpEntry *lat = modexp_entries_latency(&m);
  for (int i = 0; i < m; i++)
    if (lat[i].crt == crt) v.push_back(lat[i]);
  const ModexpEntry *small = modexp_entries_small(&m);
  for (int i = 0; i < m; i++)
    if (small[i].crt == crt) v.push_back(small[i]);
  return v;
}

const ModexpEntry *find_exact(uint32_t limbs, KernelConfig cfg, bool crt) {
  static const std::vector<ModexpEntry> full = entries(false), residue = entries(true);
  for (const ModexpEntry &e : crt ? residue : full)
    if (e.limbs == (int)limbs && e.tpi == (int)cfg.tpi && e.form == (int)cfg.form && e.table == cfg.table) return &e;
  return nullptr;
}

// The instantiation for cfg; a geometry not built with the small table runs
// with the full one (same results, only the speed differs).
const ModexpEntry *find_entry(uint32_t limbs, KernelConfig cfg, bool crt) {
  const ModexpEntry *e = find_exact(limbs, cfg, crt);
  if (e || cfg.table == kTableFull) return e;
  cfg.table = kTableFull;
  return find_exact(limbs, cfg, crt);
}

}  // namespace

int clear_status(uint32_t *status, cudaStream_t st) {
  if (cudaMemsetAsync(status, 0, 8, st) != cudaSuccess || cudaMemsetAsync(status + 2, 0xff, 8, st) != cudaSuccess)
    return PMK_ECUDA;
  return PMK_OK;
}

int launch_split(uint32_t nbits, const uint8_t *msg, size_t len, uint32_t *chunks, size_t n, cudaStream_t st) {
  const int P = (int)(nbits / 8 - 1), S = (int)(nbits / 32);
  const long long nvec = (long long)n * (S / 4);
  if (nvec == 0) return PMK_OK;
  if (reinterpret_cast<uintptr_t>(chunks) & 15u) return PMK_EINVAL;  // limb buffers are 16-byte aligned
  const int msg_aligned = (reinterpret_cast<uintptr_t>(msg) & 15u) == 0;
  const int g = grid_for(nvec, kAuxThreads);
  uint4 *out = reinterpret_cast<uint4 *>(chunks);
  if ((long long)len < (1LL << 31) && nvec < (1LL << 31))
    k_split<uint32_t><<<g, kAuxThreads, 0, st>>>(msg, (uint32_t)len, P, S, out, (uint32_t)nvec, msg_aligned,
                                                  div_magic((uint32_t)(S / 4)));
  else
    k_split<unsigned long long><<<g, kAuxThreads, 0, st>>>(msg, (unsigned long long)len, P, S, out,
                                                            (unsigned long long)nvec, msg_aligned, DivMagic{});
  return cuda_rc(cudaGetLastError());
}

int launch_join(uint32_t nbits, const uint32_t *chunks, size_t n, uint8_t *msg, size_t len, cudaStream_t st) {
  const int P = (int)(nbits / 8 - 1), S = (int)(nbits / 32);
  if (len == 0) return PMK_OK;
  if (reinterpret_cast<uintptr_t>(chunks) & 15u) return PMK_EINVAL;
  const int out_aligned = (reinterpret_cast<uintptr_t>(msg) & 15u) == 0;
  const int g = grid_for(((long long)len + 15) / 16, kAuxThreads);
  const long long nbuf16 = (long long)n * (S / 4);  // 16-byte vectors of the limb buffer
  if ((long long)len < (1LL << 31) - 16 && nbuf16 < (1LL << 31))  // 16 u stays below 2^31 (exact division)
    k_join<uint32_t><<<g, kAuxThreads, 0, st>>>(chunks, P, S, msg, (uint32_t)len, out_aligned,
                                                 div_magic((uint32_t)P), (uint32_t)nbuf16);
  else
    k_join<unsigned long long><<<g, kAuxThreads, 0, st>>>(chunks, P, S, msg, (unsigned long long)len, out_aligned,
                                                           DivMagic{}, (unsigned long long)nbuf16);
  return cuda_rc(cudaGetLastError());
}

int launch_range_check(const KeyDev *keys, uint32_t K, uint32_t s, const uint32_t *in, size_t n, uint32_t *status,
                       cudaStream_t st, const uint32_t *key_idx) {
  if (n == 0) return PMK_OK;
  k_range<<<(unsigned)((n + kAuxThreads - 1) / kAuxThreads), kAuxThreads, 0, st>>>(keys, K, (int)s, in, (long long)n,
                                                                                   status, key_idx);
  return cuda_rc(cudaGetLastError());
}

// Layout of a key-group table: poff[K + 1], slot[n + kGroupAlign K] (the
// padding of K segments is below kGroupAlign K), count[K], cursor[K].
size_t key_groups_words(size_t n, uint32_t K) {
  return (size_t)(K + 1) + (n + (size_t)kGroupAlign * K) + 2 * (size_t)K;
}

int launch_key_groups(const uint32_t *key_idx, size_t n, uint32_t K, uint32_t align, uint32_t *table,
                      uint32_t *status, cudaStream_t st) {
  if (K == 0 || K > 16383 || n >= kMaxGroupedChunks) return PMK_EINVAL;
  if (align == 0 || align > kGroupAlign || (align & (align - 1))) return PMK_EINVAL;
  const size_t nslot = n + (size_t)kGroupAlign * K;
  uint32_t *poff = table, *slot = table + K + 1, *count = slot + nslot, *cursor = count + K;
  if (cudaMemsetAsync(slot, 0xff, nslot * 4, st) != cudaSuccess ||
      cudaMemsetAsync(count, 0, (size_t)K * 4, st) != cudaSuccess)
    return PMK_ECUDA;
  if (n == 0) {
    k_key_offsets<<<1, kScanThreads, 0, st>>>(count, K, align, poff, cursor);
    return cuda_rc(cudaGetLastError());
  }
  const size_t hist_bytes = (size_t)K * 4;
  int rc = configure_smem(reinterpret_cast<const void *>(&k_key_count), 16383 * 4);  // the largest K, set once
  if (rc != PMK_OK) return rc;
  const int g = (int)std::min<long long>(grid_for((long long)n, kAuxThreads), 152LL * 4);
  k_key_count<<<g, kAuxThreads, hist_bytes, st>>>(key_idx, (long long)n, K, count, status);
  k_key_offsets<<<1, kScanThreads, 0, st>>>(count, K, align, poff, cursor);
  k_key_scatter<<<grid_for((long long)n, kAuxThreads), kAuxThreads, 0, st>>>(key_idx, (long long)n, K, cursor, slot);
  return cuda_rc(cudaGetLastError());
}

const MulmodEntry *mulmod_entries(int *count) {
  static const MulmodEntry entries[] = {
      make_mulmod<4, 2>(),   make_mulmod<8, 2>(),    make_mulmod<16, 2>(),   make_mulmod<32, 4>(),
      make_mulmod<64, 8>(),  make_mulmod<96, 8>(),   make_mulmod<128, 16>(), make_mulmod<192, 16>(),
      make_mulmod<256, 16>(),
  };
  *count = (int)(sizeof(entries) / sizeof(entries[0]));
  return entries;
}

const MulmodEntry *crt_sum_entries(int *count) {
  static const MulmodEntry entries[] = {
      make_crt_sum<4, 2>(),  make_crt_sum<8, 2>(),   make_crt_sum<16, 2>(),   make_crt_sum<32, 4>(),
      make_crt_sum<64, 8>(), make_crt_sum<96, 8>(),  make_crt_sum<128, 16>(), make_crt_sum<192, 16>(),
      make_crt_sum<256, 16>(),
  };
  *count = (int)(sizeof(entries) / sizeof(entries[0]));
  return entries;
}

int launch_crt_sum(uint32_t limbs, uint32_t parts, const KeyDev *keys, uint32_t K, uint32_t *out, size_t n,
                   cudaStream_t st, uint32_t *status_if_zero_residue, const uint32_t *groups,
                   uint32_t groups_align) {
  if (n == 0) return PMK_OK;
  if (parts < 2 || parts > (uint32_t)kMaxPrimes || limbs % parts || K == 0 || K > 65535) return PMK_EINVAL;
  int cnt = 0;
  const MulmodEntry *list = crt_sum_entries(&cnt), *e = nullptr;
  for (int i = 0; i < cnt; i++)
    if (list[i].limbs == (int)limbs) e = &list[i];
  if (!e) return PMK_EUNSUPPORTED;
  int rc = configure_smem(e->fn, e->smem);
  if (rc != PMK_OK) return rc;
  const long long per_key = ((long long)n + K - 1) / K;
  const int ipb = dev::kThreads / e->tpi;
  if (groups && (groups_align == 0 || groups_align > kGroupAlign || groups_align % ipb))
    return PMK_EUNSUPPORTED;  // a block must not straddle two keys' slots
  dim3 grid = groups ? dim3((unsigned)(((long long)n + (long long)(groups_align - 1) * K + ipb - 1) / ipb), 1)
                     : dim3((unsigned)((per_key + ipb - 1) / ipb), K);
  long long nl = (long long)n;
  int B = (int)parts;
  uint32_t *status = status_if_zero_residue;
  void *args[] = {(void *)&keys, (void *)&K, (void *)&out, (void *)&nl, (void *)&B, (void *)&status, (void *)&groups};
  return cuda_rc(cudaLaunchKernel(e->fn, grid, dim3(dev::kThreads), args, e->smem, st));
}

int launch_mulmod(uint32_t limbs, const KeyDev *keys, uint32_t K, const uint32_t *a, const uint32_t *b, uint32_t *out,
                  size_t n, cudaStream_t st) {
  if (n == 0) return PMK_OK;
  int cnt = 0;
  const MulmodEntry *list = mulmod_entries(&cnt), *e = nullptr;
  for (int i = 0; i < cnt; i++)
    if (list[i].limbs == (int)limbs) e = &list[i];
  if (!e) return PMK_EUNSUPPORTED;
  int rc = configure_smem(e->fn, e->smem);
  if (rc != PMK_OK) return rc;
  const long long per_key = ((long long)n + K - 1) / K;
  const int ipb = dev::kThreads / e->tpi;
  dim3 grid((unsigned)((per_key + ipb - 1) / ipb), K);
  long long nl = (long long)n;
  void *args[] = {(void *)&keys, (void *)&K, (void *)&a, (void *)&b, (void *)&out, (void *)&nl};
  return cuda_rc(cudaLaunchKernel(e->fn, grid, dim3(dev::kThreads), args, e->smem, st));
}

int launch_modexp_naive(bool enc, uint32_t limbs, const KeyDev *keys, uint32_t K, const uint32_t *in, uint32_t *out,
                        size_t n, cudaStream_t st) {
  if (n == 0) return PMK_OK;
  const unsigned blocks = (unsigned)((n + 127) / 128);
  const int e = enc ? 1 : 0;
  switch (limbs) {
    case 32: k_modexp_naive<32><<<blocks, 128, 0, st>>>(keys, K, in, out, (long long)n, e); break;
    case 64: k_modexp_naive<64><<<blocks, 128, 0, st>>>(keys, K, in, out, (long long)n, e); break;
    default: return PMK_EUNSUPPORTED;
  }
  return cuda_rc(cudaGetLastError());
}

bool modexp_built(uint32_t limbs, KernelConfig cfg, bool crt) { return find_entry(limbs, cfg, crt) != nullptr; }

uint32_t modexp_block_instances(uint32_t limbs, KernelConfig cfg, bool crt) {
  const ModexpEntry *e = find_entry(limbs, cfg, crt);
  return e ? (uint32_t)(e->threads / e->tpi) : 0u;
}

uint32_t crt_sum_block_instances(uint32_t limbs) {
  int cnt = 0;
  const MulmodEntry *list = crt_sum_entries(&cnt);
  for (int i = 0; i < cnt; i++)
    if (list[i].limbs == (int)limbs) return (uint32_t)(dev::kThreads / list[i].tpi);
  return 0u;
}

// Defaults measured on GB300 (1 MiB and 100 MiB workloads at 2048 bits):
// 64-limb full-width and 32-limb CRT residues run fastest with independent
// columns at 8 and 4 lanes; other widths use the carry-chain form.
KernelConfig default_config(uint32_t limbs, bool crt) {
  KernelConfig c;
  switch (limbs) {
    case 2: case 4: case 8: case 16: c.tpi = 2; break;
    case 32: c.tpi = 4; c.form = crt ? 1 : 0; break;
    case 48: case 96: c.tpi = 8; break;
    case 64: c.tpi = 8; c.form = crt ? 0 : 1; break;
    case 128: case 192: case 256: c.tpi = 16; break;
    default: break;
  }
  if (c.tpi && !find_entry(limbs, c, crt)) c = KernelConfig();
  return c;
}

int list_configs(uint32_t limbs, bool crt, KernelConfig *out, int max) {
  int k = 0;
  const std::vector<ModexpEntry> all = entries(crt);
  for (size_t i = 0; i < all.size(); i++) {
    const ModexpEntry &e = all[i];
    if (e.limbs != (int)limbs || e.table != kTableFull) continue;  // geometries; small-table twins are not listed
    bool seen = false;  // block-size twins are one geometry
    for (size_t j = 0; j < i && !seen; j++)
      seen = all[j].limbs == e.limbs && all[j].tpi == e.tpi && all[j].form == e.form && all[j].table == kTableFull;
    if (seen) continue;
    if (k < max && out) out[k] = KernelConfig{(uint32_t)e.tpi, (uint32_t)e.form};
    k++;
  }
  return k;
}

// Raise a kernel's dynamic shared-memory limit once per device.
int configure_smem(const void *fn, size_t bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void *, int>> done;
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PMK_ECUDA;
  if (!done.count({fn, dev})) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
      return PMK_ECUDA;
    done.insert({fn, dev});
  }
  return PMK_OK;
}

int modexp_tasks_blocks_per_sm(uint32_t limbs, KernelConfig cfg, bool crt) {
  const ModexpEntry *e = find_entry(limbs, cfg, crt);
  if (!e || configure_smem(e->fn_tasks, e->smem_tasks) != PMK_OK) return 0;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, e->fn_tasks, dev::kThreads, e->smem_tasks) != cudaSuccess)
    return 0;
  return blocks;
}

bool modexp_small_table_built(uint32_t limbs, KernelConfig cfg, bool crt) {
  cfg.table = kTableSmall;
  return find_exact(limbs, cfg, crt) != nullptr;
}

long long modexp_resident_instances(uint32_t limbs, KernelConfig cfg, bool crt) {
  const int per_sm = modexp_tasks_blocks_per_sm(limbs, cfg, crt);
  int dev = 0, sms = 0;
  if (per_sm <= 0 || cfg.tpi == 0 || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return (long long)per_sm * sms * (dev::kThreads / (int)cfg.tpi);
}

int launch_modexp_tasks(uint32_t limbs, KernelConfig cfg, bool crt, const BatchTask *tasks, int ntasks, int *counter,
                        int blocks, cudaStream_t st) {
  if (ntasks == 0) return PMK_OK;
  const ModexpEntry *e = find_entry(limbs, cfg, crt);
  if (!e) return PMK_EUNSUPPORTED;
  int rc = configure_smem(e->fn_tasks, e->smem_tasks);
  if (rc != PMK_OK) return rc;
  void *args[] = {(void *)&tasks, (void *)&ntasks, (void *)&counter};
  return cuda_rc(cudaLaunchKernel(e->fn_tasks, dim3(blocks), dim3(dev::kThreads), args, e->smem_tasks, st));
}

int launch_modexp(ExpMode mode, uint32_t limbs, KernelConfig cfg, const KeyDev *keys, uint32_t K, const uint32_t *in,
                  uint32_t *out, size_t n, cudaStream_t st, uint32_t parts, const uint32_t *groups,
                  uint32_t groups_align) {
  if (n == 0) return PMK_OK;
  const bool crt = mode == ExpMode::kCrtHalf || mode == ExpMode::kCrtInverse;
  if (crt && (parts < 2 || parts > (uint32_t)kMaxPrimes)) return PMK_EINVAL;
  if (!groups && (unsigned long long)K * (crt ? parts : 1) > 65535ull) return PMK_EINVAL;  // grid.y
  const ModexpEntry *e = find_entry(limbs, cfg, crt);
  if (!e) return PMK_EUNSUPPORTED;
  const void *fn = groups ? e->fn_grp : e->fn;
  const int rc = configure_smem(fn, e->smem);
  if (rc != PMK_OK) return rc;
  const long long per_key = ((long long)n + K - 1) / K;
  const int ipb = e->threads / e->tpi;
  if (groups && (groups_align == 0 || groups_align > kGroupAlign || groups_align % ipb))
    return PMK_EUNSUPPORTED;  // a block must not straddle two keys' slots
  dim3 grid = groups ? dim3((unsigned)(((long long)n + (long long)(groups_align - 1) * K + ipb - 1) / ipb), crt ? parts : 1)
                     : dim3((unsigned)((per_key + ipb - 1) / ipb), crt ? parts * K : K);
  long long nl = (long long)n;
  int sel = (mode == ExpMode::kEncrypt || mode == ExpMode::kCrtInverse) ? 1 : 0;
  int np = crt ? (int)parts : 1;
  void *args[] = {(void *)&keys, (void *)&K,   (void *)&in, (void *)&out,
                  (void *)&nl,   (void *)&sel, (void *)&np, (void *)&groups};
  return cuda_rc(cudaLaunchKernel(fn, grid, dim3(e->threads), args, e->smem, st));
}

}  // namespace pmk
