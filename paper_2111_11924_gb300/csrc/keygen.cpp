// Host key initialisation for PMKRSA (Section 1.1 steps 1a-1c and Algorithm 1
// "Initialization"), the Montgomery constants the kernels need, and the
// sliding-window exponent schedules.
//
// Arithmetic here is the library's own: 64-bit limbs with 128-bit products,
// Montgomery multiplication for Miller-Rabin and Fermat inversion, and the
// small-exponent identity d = (k phi + 1) / e for the private exponent.  It
// needs no general division routine.
//
// Reading of the unspecified parts of key generation (the paper draws from
// /dev/random, Section 3.3): SplitMix64 (Steele, Lea, Flood 2014); key k uses
// its own stream seeded by the k-th output of a master stream seeded by the
// caller, so keys are generated in parallel (Section 3.3 uses OpenMP).  A
// prime candidate is nbits/128 SplitMix64 words, little-endian, with its top
// two bits and bit 0 set; it is rejected if an odd prime below 2000 divides
// it, then if gcd(e, cand - 1) != 1, then by 40 Miller-Rabin rounds with bases
// (splitmix64() >> 1) + 2.  q is redrawn while q == p.
//
// Multi-prime keys (Section 2.1): b primes of nbits / b bits drawn in order
// from the key's stream, each redrawn while it equals an earlier one; a
// candidate is also redrawn while its top byte is below the least T with
// T^b >= 2^(8b - 1), so that N has exactly nbits bits (T = 192 for b = 2:
// the two-top-bits rule above, so b = 2 gives the same keys).
#include <algorithm>
#include <cstring>
#include <thread>

#include "pmk_internal.h"

namespace pmk {
namespace {

using u64 = uint64_t;
using u128 = unsigned __int128;

u64 splitmix64(u64 &state) {
  u64 z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ---- fixed-width unsigned arithmetic on n 64-bit limbs ----

int cmp(const u64 *a, const u64 *b, int n) {
  for (int i = n - 1; i >= 0; i--)
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  return 0;
}

u64 sub(u64 *r, const u64 *a, const u64 *b, int n) {
  u64 borrow = 0;
  for (int i = 0; i < n; i++) {
    u128 d = (u128)a[i] - b[i] - borrow;
    r[i] = (u64)d;
    borrow = (u64)(d >> 127);
  }
  return borrow;
}

u64 mod_small(const u64 *a, int n, u64 m) {
  u128 r = 0;
  for (int i = n - 1; i >= 0; i--) r = ((r << 64) | a[i]) % m;
  return (u64)r;
}

// r = 2 r mod m (r < m)
void dbl_mod(u64 *r, const u64 *m, int n) {
  u64 top = r[n - 1] >> 63;
  for (int i = n - 1; i > 0; i--) r[i] = (r[i] << 1) | (r[i - 1] >> 63);
  r[0] <<= 1;
  if (top || cmp(r, m, n) >= 0) sub(r, r, m, n);
}

// Montgomery arithmetic modulo an odd m with R = 2^(64 n).
struct Mont {
  int n;
  std::vector<u64> m, r2;  // r2 = R^2 mod m
  u64 m0inv;               // -m^-1 mod 2^64
  explicit Mont(const std::vector<u64> &mod) : n((int)mod.size()), m(mod), r2(mod.size(), 0) {
    u64 inv = m[0];  // Newton: inv = m^-1 mod 2^64
    for (int i = 0; i < 6; i++) inv *= 2 - m[0] * inv;
    m0inv = (u64)0 - inv;
    r2[0] = 1;
    for (int i = 0; i < 128 * n; i++) dbl_mod(r2.data(), m.data(), n);
  }
  // out = a b R^-1 mod m  (CIOS, a, b < m)
  void mul(u64 *out, const u64 *a, const u64 *b) const {
    std::vector<u64> t(n + 2, 0);
    for (int i = 0; i < n; i++) {
      u128 c = 0;
      for (int j = 0; j < n; j++) {
        c += (u128)a[j] * b[i] + t[j];
        t[j] = (u64)c;
        c >>= 64;
      }
      c += t[n];
      t[n] = (u64)c;
      t[n + 1] = (u64)(c >> 64);
      u64 q = t[0] * m0inv;
      c = ((u128)q * m[0] + t[0]) >> 64;
      for (int j = 1; j < n; j++) {
        c += (u128)q * m[j] + t[j];
        t[j - 1] = (u64)c;
        c >>= 64;
      }
      c += t[n];
      t[n - 1] = (u64)c;
      t[n] = t[n + 1] + (u64)(c >> 64);
    }
    if (t[n] || cmp(t.data(), m.data(), n) >= 0) sub(t.data(), t.data(), m.data(), n);
    std::memcpy(out, t.data(), sizeof(u64) * n);
  }
  void to_mont(u64 *out, const u64 *a) const { mul(out, a, r2.data()); }
  void from_mont(u64 *out, const u64 *a) const {
    std::vector<u64> one(n, 0);
    one[0] = 1;
    mul(out, a, one.data());
  }
  // out = b^x mod m, plain left-to-right binary over the bits of x (nx limbs)
  void pow(u64 *out, const u64 *b, const u64 *x, int nx) const {
    std::vector<u64> base(n), acc(n), one(n, 0);
    one[0] = 1;
    to_mont(base.data(), b);
    to_mont(acc.data(), one.data());
    for (int i = 64 * nx - 1; i >= 0; i--) {
      mul(acc.data(), acc.data(), acc.data());
      if ((x[i / 64] >> (i % 64)) & 1) mul(acc.data(), acc.data(), base.data());
    }
    from_mont(out, acc.data());
  }
};

bool miller_rabin_round(const Mont &mt, u64 base) {
  int n = mt.n;
  std::vector<u64> n1(mt.m), one(n, 0), d(n), x(n), b(n, 0);
  one[0] = 1;
  sub(n1.data(), mt.m.data(), one.data(), n);
  int s = 0;
  while (!((n1[s / 64] >> (s % 64)) & 1)) s++;
  for (int i = 0; i < n; i++) {  // d = (m - 1) >> s
    int bit = s + 64 * i, w = bit / 64, sh = bit % 64;
    u64 lo = w < n ? n1[w] >> sh : 0;
    u64 hi = (w + 1 < n && sh) ? n1[w + 1] << (64 - sh) : 0;
    d[i] = lo | hi;
  }
  b[0] = base;
  mt.pow(x.data(), b.data(), d.data(), n);
  if (cmp(x.data(), one.data(), n) == 0 || cmp(x.data(), n1.data(), n) == 0) return true;
  std::vector<u64> xm(n), n1m(n);
  mt.to_mont(xm.data(), x.data());
  mt.to_mont(n1m.data(), n1.data());
  std::vector<u64> onem(n);
  mt.to_mont(onem.data(), one.data());
  for (int i = 1; i < s; i++) {
    mt.mul(xm.data(), xm.data(), xm.data());
    if (cmp(xm.data(), n1m.data(), n) == 0) return true;
    if (cmp(xm.data(), onem.data(), n) == 0) return false;
  }
  return false;
}

u64 gcd64(u64 a, u64 b) {
  while (b) {
    u64 t = a % b;
    a = b;
    b = t;
  }
  return a;
}

const std::vector<u64> &small_primes() {
  static const std::vector<u64> primes = [] {
    std::vector<bool> comp(2000, false);
    std::vector<u64> v;
    for (int i = 2; i < 2000; i++) {
      if (comp[i]) continue;
      if (i > 2) v.push_back(i);
      for (int j = i * i; j < 2000; j += i) comp[j] = true;
    }
    return v;
  }();
  return primes;
}

// A prime of exactly `bits` bits whose top byte is at least min_top (>= 192).
std::vector<u64> gen_prime(u64 &rng, int bits, u64 e, int min_top) {
  int n = bits / 64;
  std::vector<u64> p(n);
  for (;;) {
    for (int w = 0; w < n; w++) p[w] = splitmix64(rng);
    p[n - 1] |= 0xC000000000000000ull;
    p[0] |= 1;
    if ((int)(p[n - 1] >> 56) < min_top) continue;
    bool composite = false;
    for (u64 sp : small_primes())
      if (mod_small(p.data(), n, sp) == 0) {
        composite = true;
        break;
      }
    if (composite) continue;
    u64 r = mod_small(p.data(), n, e);           // (p - 1) mod e
    r = (r + e - 1) % e;
    if (gcd64(e, r) != 1) continue;
    Mont mt(p);
    bool ok = true;
    for (int round = 0; round < 40 && ok; round++) ok = miller_rabin_round(mt, (splitmix64(rng) >> 1) + 2);
    if (ok) return p;
  }
}

// inverse of a modulo m (gcd 1), small word-size values
u64 inv_small(u64 a, u64 m) {
  __int128 t0 = 0, t1 = 1, r0 = m, r1 = a % m;
  while (r1) {
    __int128 q = r0 / r1, tmp;
    tmp = r0 - q * r1; r0 = r1; r1 = tmp;
    tmp = t0 - q * t1; t0 = t1; t1 = tmp;
  }
  if (t0 < 0) t0 += m;
  return (u64)t0;
}

// x^-1 mod phi for a small x (here the public exponent), via
// x^-1 = (k phi + 1) / x with k = -phi^-1 mod x.  phi has n limbs.
std::vector<u64> inv_of_small(u64 x, const std::vector<u64> &phi) {
  int n = (int)phi.size();
  u64 k = (x - inv_small(mod_small(phi.data(), n, x), x)) % x;
  std::vector<u64> t(n + 1, 0);
  u128 c = 1;  // t = k phi + 1
  for (int i = 0; i < n; i++) {
    c += (u128)k * phi[i];
    t[i] = (u64)c;
    c >>= 64;
  }
  t[n] = (u64)c;
  u128 rem = 0;  // exact division by x
  for (int i = n; i >= 0; i--) {
    u128 cur = (rem << 64) | t[i];
    t[i] = (u64)(cur / x);
    rem = cur % x;
  }
  t.resize(n);
  return t;
}

std::vector<uint32_t> to32(const std::vector<u64> &a, size_t nlimbs32) {
  std::vector<uint32_t> r(nlimbs32, 0);
  for (size_t i = 0; i < a.size() && 2 * i < nlimbs32; i++) {
    r[2 * i] = (uint32_t)a[i];
    if (2 * i + 1 < nlimbs32) r[2 * i + 1] = (uint32_t)(a[i] >> 32);
  }
  return r;
}

std::vector<u64> to64(const uint32_t *a, size_t nlimbs32) {
  std::vector<u64> r((nlimbs32 + 1) / 2, 0);
  for (size_t i = 0; i < nlimbs32; i++) r[i / 2] |= (u64)a[i] << (32 * (i % 2));
  return r;
}

std::vector<u64> mul_full(const std::vector<u64> &a, const std::vector<u64> &b) {
  std::vector<u64> r(a.size() + b.size(), 0);
  for (size_t i = 0; i < b.size(); i++) {
    u128 c = 0;
    for (size_t j = 0; j < a.size(); j++) {
      c += (u128)a[j] * b[i] + r[i + j];
      r[i + j] = (u64)c;
      c >>= 64;
    }
    r[i + a.size()] = (u64)c;
  }
  return r;
}

std::vector<u64> minus_one(std::vector<u64> a) {
  for (auto &w : a)
    if (w-- != 0) break;
  return a;
}

uint32_t neg_inv32(uint32_t m0) {
  uint32_t inv = m0;
  for (int i = 0; i < 5; i++) inv *= 2 - m0 * inv;
  return 0u - inv;
}

// 2^(32 k) mod m for k = ks[...], by repeated doubling (m odd, n limbs)
void pow2_mod(const std::vector<u64> &m, int bits_a, int bits_b, std::vector<u64> &ra, std::vector<u64> &rb) {
  int n = (int)m.size();
  std::vector<u64> r(n, 0);
  r[0] = 1;
  for (int i = 1; i <= std::max(bits_a, bits_b); i++) {
    dbl_mod(r.data(), m.data(), n);
    if (i == bits_a) ra = r;
    if (i == bits_b) rb = r;
  }
}

// x mod m for x < 2 m (one conditional subtraction), n limbs
std::vector<u64> reduce_once(std::vector<u64> x, const std::vector<u64> &m) {
  const int n = (int)m.size();
  if (cmp(x.data(), m.data(), n) >= 0) sub(x.data(), x.data(), m.data(), n);
  return x;
}

// 2^(32 k) mod m as 32-bit limbs, for the Montgomery constants R^2, R^3.
std::vector<uint32_t> pow2_32(const std::vector<u64> &m, int k, size_t limbs) {
  std::vector<u64> a, unused;
  pow2_mod(m, k, k, a, unused);
  return to32(a, limbs);
}

// Key data for primes r_0 .. r_{b-1} of equal size (b >= 2).  Every prime's
// top byte is >= 192, so r_j < 2 r_i for all i, j: a prime reduces modulo
// another by one conditional subtraction.
void finish_key(uint32_t nbits, u64 e, const std::vector<std::vector<u64>> &r, HostKey &k) {
  const int b = (int)r.size(), n = (int)r[0].size();
  const size_t s = nbits / 32, h = s / b;
  std::vector<u64> N = r[0], phi = minus_one(r[0]);
  for (int i = 1; i < b; i++) {
    N = mul_full(N, r[i]);
    phi = mul_full(phi, minus_one(r[i]));
  }
  N.resize(s / 2);
  phi.resize(s / 2);
  const std::vector<u64> d = inv_of_small(e, phi);
  std::vector<u64> two(n, 0);
  two[0] = 2;
  k.nprimes = (uint32_t)b;
  k.N = to32(N, s);
  k.d = to32(d, s);
  k.n0 = neg_inv32(k.N[0]);
  k.R2 = pow2_32(N, (int)(64 * s), s);
  for (int i = 0; i < b; i++) {
    const Mont mt(r[i]);
    std::vector<u64> rm2(r[i]);
    sub(rm2.data(), r[i].data(), two.data(), n);
    k.pr[i] = to32(r[i], h);
    k.dpr[i] = to32(inv_of_small(e, minus_one(r[i])), h);  // = d mod (r_i - 1)
    k.n0h[i] = neg_inv32(k.pr[i][0]);
    k.R2h[i] = pow2_32(r[i], (int)(64 * h), h);
    k.R3h[i] = pow2_32(r[i], (int)(96 * h), h);
    const std::vector<uint32_t> rm2_32 = to32(rm2, h);
    for (int t = 0; t < 2; t++) {
      k.sched_h[t][i] = make_schedule(k.dpr[i].data(), (int)h, window_of(t));
      k.sched_hinv[t][i] = make_schedule(rm2_32.data(), (int)h, window_of(t));
    }
    {  // blinded CRT: exponents d_i and r_i - 1 - d_i
      std::vector<u64> eb = minus_one(r[i]), di = to64(k.dpr[i].data(), h);
      sub(eb.data(), eb.data(), di.data(), n);
      const std::vector<uint32_t> eb32 = to32(eb, h);
      k.sched_blind[i] = make_schedule2(k.dpr[i].data(), eb32.data(), (int)h);
    }
    if (i == 1) continue;
    // Garner coefficients (exported): coef_0 = r_1^-1 mod r_0,
    // coef_i = (r_0 ... r_{i-1})^-1 mod r_i, by Fermat
    std::vector<u64> acc(n), t(n), x(n), coef(n);
    bool first = true;
    for (int j = 0; j < b; j++) {
      const bool before = i == 0 ? j == 1 : j < i;
      if (!before) continue;
      mt.to_mont(t.data(), reduce_once(r[j], r[i]).data());
      if (first) acc = t;
      else mt.mul(acc.data(), acc.data(), t.data());
      first = false;
    }
    mt.from_mont(x.data(), acc.data());
    mt.pow(coef.data(), x.data(), rm2.data(), n);
    k.coef[i] = to32(coef, h);
  }
  // CRT recombination rows c_i R mod N, c_i = (N / r_i) ((N / r_i)^-1 mod r_i)
  const Mont mN(N);
  for (int i = 0; i < b; i++) {
    const Mont mt(r[i]);
    std::vector<u64> others, acc(n), t(n), x(n), inv(n), rm2(r[i]);
    sub(rm2.data(), r[i].data(), two.data(), n);
    bool first = true;
    for (int j = 0; j < b; j++) {
      if (j == i) continue;
      others = others.empty() ? r[j] : mul_full(others, r[j]);
      mt.to_mont(t.data(), reduce_once(r[j], r[i]).data());
      if (first) acc = t;
      else mt.mul(acc.data(), acc.data(), t.data());
      first = false;
    }
    mt.from_mont(x.data(), acc.data());
    mt.pow(inv.data(), x.data(), rm2.data(), n);     // (N / r_i)^-1 mod r_i (Fermat)
    std::vector<u64> c = mul_full(others, inv), cR(s / 2);
    c.resize(s / 2);                                   // c_i < N
    mN.to_mont(cR.data(), c.data());
    k.crt_sum[i] = to32(cR, s);
  }
  k.p = k.pr[0];
  k.q = k.pr[1];
  k.dp = k.dpr[0];
  k.dq = k.dpr[1];
  k.qinv = k.coef[0];
  uint32_t ev[2] = {(uint32_t)e, (uint32_t)(e >> 32)};
  for (int t = 0; t < 2; t++) {
    k.sched_e[t] = make_schedule(ev, 2, window_of(t));
    k.sched_d[t] = make_schedule(k.d.data(), (int)s, window_of(t));
  }
}

// The least top byte T (at least 192) with T^b >= 2^(8 b - 1): b primes of
// k bits whose top bytes are >= T multiply to at least 2^(b k - 1).
int min_top_byte(int b) {
  const u64 need = 1ull << (8 * b - 1);
  int t = 192;
  for (;; t++) {
    u64 v = 1;
    for (int i = 0; i < b; i++) v *= (u64)t;
    if (v >= need) return t;
  }
}

bool valid_width(uint32_t nbits) { return nbits >= 128 && nbits <= 8192 && nbits % 128 == 0; }

}  // namespace

// Sliding-window recoding of an exponent, scanned from its top bit.  The
// window width w <= max_window (a table of 2^(max_window - 1) odd powers)
// minimises the product count (table entries + multiplies) for this exponent.
Schedule make_schedule(const uint32_t *exp, int nlimbs, uint32_t max_window) {
  int top = -1;
  for (int i = 32 * nlimbs - 1; i >= 0; i--)
    if ((exp[i / 32] >> (i % 32)) & 1) {
      top = i;
      break;
    }
  Schedule best;
  size_t best_cost = ~(size_t)0;
  if (top < 0) return best;  // exponent 0: empty schedule (callers reject it)
  auto bit = [&](int i) { return (exp[i / 32] >> (i % 32)) & 1; };
  for (int w = 1; w <= (int)max_window; w++) {
    Schedule sc;
    int i = top, pending = 0;
    bool first = true;
    size_t muls = 0;
    while (i >= 0) {
      if (!bit(i)) {
        pending++;
        i--;
        continue;
      }
      int j = std::max(i - w + 1, 0);
      while (!bit(j)) j++;
      uint32_t v = 0;
      for (int b = i; b >= j; b--) v = (v << 1) | bit(b);
      uint32_t idx = (v - 1) / 2;
      if (first) {
        sc.steps.push_back(idx);
        first = false;
      } else {
        sc.steps.push_back(((uint32_t)(pending + (i - j + 1)) << 8) | idx);
        muls++;
      }
      sc.maxidx = std::max(sc.maxidx, idx);
      pending = 0;
      i = j - 1;
    }
    if (pending) sc.steps.push_back(((uint32_t)pending << 8) | 0xFFu);
    size_t cost = muls + sc.maxidx + (sc.maxidx ? 1 : 0);
    if (cost < best_cost) {
      best_cost = cost;
      best = sc;
    }
  }
  return best;
}

bool valid_multiprime(uint32_t nbits, uint32_t nprimes) {
  return nprimes >= 2 && nprimes <= (uint32_t)kMaxPrimes && valid_width(nbits) && nbits % (64 * nprimes) == 0;
}

namespace {

// Left-to-right sliding windows of width <= w over exp: (lowest bit, odd-power index).
std::vector<std::pair<int, uint32_t>> sliding_windows(const uint32_t *exp, int nlimbs, int w) {
  std::vector<std::pair<int, uint32_t>> out;
  auto bit = [&](int i) { return (exp[i / 32] >> (i % 32)) & 1; };
  int i = 32 * nlimbs - 1;
  while (i >= 0) {
    if (!bit(i)) {
      i--;
      continue;
    }
    int j = std::max(i - w + 1, 0);
    while (!bit(j)) j++;
    uint32_t v = 0;
    for (int b = i; b >= j; b--) v = (v << 1) | bit(b);
    out.push_back({j, (v - 1) / 2});
    i = j - 1;
  }
  return out;
}

// Windows of width <= 4 (8 odd powers) that minimise windows + table products.
std::vector<std::pair<int, uint32_t>> best_windows(const uint32_t *exp, int nlimbs, uint32_t *maxidx) {
  std::vector<std::pair<int, uint32_t>> best;
  size_t best_cost = ~(size_t)0;
  for (int w = 1; w <= 4; w++) {
    auto ws = sliding_windows(exp, nlimbs, w);
    uint32_t mx = 0;
    for (auto &x : ws) mx = std::max(mx, x.second);
    const size_t cost = ws.size() + mx + (mx ? 1 : 0);
    if (cost < best_cost) {
      best_cost = cost;
      best = ws;
      *maxidx = mx;
    }
  }
  return best;
}

}  // namespace

Schedule2 make_schedule2(const uint32_t *expa, const uint32_t *expb, int nlimbs) {
  Schedule2 sc;
  auto wa = best_windows(expa, nlimbs, &sc.maxa);
  auto wb = best_windows(expb, nlimbs, &sc.maxb);
  if (wa.empty() || wb.empty()) return Schedule2();  // a zero exponent: callers reject it
  struct Ev {
    int pos, which;
    uint32_t idx;
  };
  std::vector<Ev> ev;
  for (auto &x : wa) ev.push_back({x.first, 0, x.second});
  for (auto &x : wb) ev.push_back({x.first, 1, x.second});
  std::stable_sort(ev.begin(), ev.end(), [](const Ev &x, const Ev &y) { return x.pos > y.pos; });
  int prev = -1;
  for (size_t k = 0; k < ev.size();) {
    const int p = ev[k].pos;
    uint32_t ia = 0xFF, ib = 0xFF;
    for (; k < ev.size() && ev[k].pos == p; k++) (ev[k].which == 0 ? ia : ib) = ev[k].idx;
    const uint32_t nsq = prev < 0 ? 0u : (uint32_t)(prev - p);
    sc.steps.push_back((nsq << 16) | (ia << 8) | ib);
    prev = p;
  }
  if (prev > 0) sc.steps.push_back(((uint32_t)prev << 16) | 0xFFFFu);
  return sc;
}

int host_keygen_mp(uint32_t K, uint32_t nbits, uint32_t nprimes, uint64_t e, uint64_t seed,
                   std::vector<HostKey> &out) {
  if (K == 0 || !valid_multiprime(nbits, nprimes) || e < 3 || !(e & 1) || e >> 32) return PMK_EINVAL;
  std::vector<u64> seeds(K);
  u64 master = seed;
  for (uint32_t k = 0; k < K; k++) seeds[k] = splitmix64(master);
  out.assign(K, HostKey());
  const int top = min_top_byte((int)nprimes), bits = (int)(nbits / nprimes);
  auto work = [&](uint32_t k) {
    u64 rng = seeds[k];
    std::vector<std::vector<u64>> r;
    for (uint32_t i = 0; i < nprimes; i++) {
      std::vector<u64> c;
      bool dup;
      do {  // r_i is redrawn while it equals an earlier prime
        c = gen_prime(rng, bits, e, top);
        dup = false;
        for (const auto &x : r) dup = dup || cmp(x.data(), c.data(), (int)c.size()) == 0;
      } while (dup);
      r.push_back(c);
    }
    finish_key(nbits, e, r, out[k]);
  };
  unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  unsigned nt = std::min<unsigned>(hw, K);
  std::vector<std::thread> pool;
  for (unsigned t = 0; t < nt; t++)
    pool.emplace_back([&, t] {
      for (uint32_t k = t; k < K; k += nt) work(k);
    });
  for (auto &th : pool) th.join();
  return PMK_OK;
}

int host_keygen(uint32_t K, uint32_t nbits, uint64_t e, uint64_t seed, std::vector<HostKey> &out) {
  return host_keygen_mp(K, nbits, 2, e, seed, out);
}

int host_from_primes(uint32_t nbits, uint64_t e, const uint32_t *p32, const uint32_t *q32, HostKey &out) {
  if (!valid_width(nbits) || e < 3 || !(e & 1) || e >> 32) return PMK_EINVAL;
  size_t h = nbits / 64;
  std::vector<u64> p = to64(p32, h), q = to64(q32, h);
  int n = (int)p.size();
  for (const auto *f : {&p, &q}) {
    if (!((*f)[0] & 1) || ((*f)[n - 1] >> 62) != 3) return PMK_EINVAL;
    u64 r = (mod_small(f->data(), n, e) + e - 1) % e;
    if (gcd64(e, r) != 1) return PMK_EINVAL;
  }
  if (cmp(p.data(), q.data(), n) == 0) return PMK_EINVAL;
  finish_key(nbits, e, {p, q}, out);
  return PMK_OK;
}

int host_from_primes_mp(uint32_t nbits, uint32_t nprimes, uint64_t e, const uint32_t *primes32, HostKey &out) {
  if (!valid_multiprime(nbits, nprimes) || e < 3 || !(e & 1) || e >> 32) return PMK_EINVAL;
  const size_t h = nbits / 32 / nprimes;
  std::vector<std::vector<u64>> r;
  for (uint32_t i = 0; i < nprimes; i++) {
    std::vector<u64> f = to64(primes32 + i * h, h);
    const int n = (int)f.size();
    if (!(f[0] & 1) || (f[n - 1] >> 62) != 3) return PMK_EINVAL;  // odd, exactly nbits/b bits, top two set
    const u64 rm = (mod_small(f.data(), n, e) + e - 1) % e;
    if (gcd64(e, rm) != 1) return PMK_EINVAL;
    for (const auto &x : r)
      if (cmp(x.data(), f.data(), n) == 0) return PMK_EINVAL;
    r.push_back(f);
  }
  std::vector<u64> N = r[0];
  for (uint32_t i = 1; i < nprimes; i++) N = mul_full(N, r[i]);
  if (!(N[N.size() - 1] >> 63)) return PMK_EINVAL;  // the modulus must have exactly nbits bits
  finish_key(nbits, e, r, out);
  return PMK_OK;
}

}  // namespace pmk
