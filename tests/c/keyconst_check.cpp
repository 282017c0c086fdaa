// Host check of the per-key constants that the kernels use but the C ABI
// does not export, on keys whose primes fit in 64 bits (128-bit moduli with
// two primes and 256-bit moduli with four; the code is the same at every
// width).  Each value is recomputed here from its definition with 128-bit
// integer arithmetic, independently of the library's own bignum:
//   N = r_0 ... r_{b-1};  n0 = -N^-1 mod 2^32;  R^2 mod N (checked modulo
//   every prime, and below N);  per prime R_h^2, R_h^3 mod r_i,
//   -r_i^-1 mod 2^32, e (d mod (r_i - 1)) = 1 mod (r_i - 1);
//   the Garner coefficients (Section 2.1): coef_0 r_1 = 1 mod r_0,
//   coef_1 = 0, coef_i r_0 ... r_{i-1} = 1 mod r_i;
//   the recombination rows c_i R mod N: below N, and = R mod r_j when
//   j = i, 0 mod r_j otherwise (c_i = 1 mod r_i, 0 mod the other primes).
// Built with g++ against keygen.cpp; no GPU.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "pmk_internal.h"

namespace {

using u128 = unsigned __int128;
using Big = std::vector<uint32_t>;

uint64_t as64(const Big &x) {
  uint64_t v = 0;
  for (size_t i = x.size(); i-- > 0;) v = (v << 32) | x[i];
  return v;
}

uint64_t mod64(const Big &x, uint64_t m) {  // Horner over the limbs
  u128 r = 0;
  for (size_t i = x.size(); i-- > 0;) r = ((r << 32) | x[i]) % m;
  return (uint64_t)r;
}

uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((u128)a * b % m); }

uint64_t pow2mod(uint64_t k, uint64_t m) {  // 2^k mod m
  uint64_t r = 1 % m, b = 2 % m;
  for (; k; k >>= 1, b = mulmod(b, b, m))
    if (k & 1) r = mulmod(r, b, m);
  return r;
}

Big mul_small(const Big &x, uint64_t v) {  // x * v, exact
  Big out(x.size() + 2, 0);
  u128 c = 0;
  for (size_t i = 0; i < out.size(); i++) {
    const u128 t = (i < x.size() ? (u128)x[i] * v : 0) + c;
    out[i] = (uint32_t)t;
    c = t >> 32;
  }
  return out;
}

bool equal_value(const Big &a, const Big &b) {
  const size_t n = a.size() > b.size() ? a.size() : b.size();
  for (size_t i = 0; i < n; i++)
    if ((i < a.size() ? a[i] : 0u) != (i < b.size() ? b[i] : 0u)) return false;
  return true;
}

bool less(const Big &a, const Big &b) {
  const size_t n = a.size() > b.size() ? a.size() : b.size();
  for (size_t i = n; i-- > 0;) {
    const uint32_t x = i < a.size() ? a[i] : 0u, y = i < b.size() ? b[i] : 0u;
    if (x != y) return x < y;
  }
  return false;
}

int g_failures = 0, g_checks = 0;

void expect(bool ok, const char *what, uint32_t nbits, uint32_t b, int key) {
  g_checks++;
  if (!ok && g_failures++ < 20) std::printf("FAIL %s (nbits %u, primes %u, key %d)\n", what, nbits, b, key);
}

void check_keys(uint32_t K, uint32_t nbits, uint32_t b, uint64_t e, uint64_t seed) {
  std::vector<pmk::HostKey> keys;
  const int rc = pmk::host_keygen_mp(K, nbits, b, e, seed, keys);
  expect(rc == PMK_OK && keys.size() == K, "keygen", nbits, b, -1);
  const uint32_t s = nbits / 32, h = s / b;
  for (uint32_t k = 0; k < keys.size(); k++) {
    const pmk::HostKey &key = keys[k];
    const int kk = (int)k;
    expect(key.nprimes == b, "prime count", nbits, b, kk);
    std::vector<uint64_t> r(b);
    for (uint32_t i = 0; i < b; i++) r[i] = as64(key.pr[i]);
    Big prod(1, 1);
    for (uint32_t i = 0; i < b; i++) prod = mul_small(prod, r[i]);
    expect(equal_value(prod, key.N), "N = product of the primes", nbits, b, kk);
    expect((uint32_t)(key.n0 * key.N[0]) == 0xFFFFFFFFu, "n0 = -N^-1 mod 2^32", nbits, b, kk);
    expect(less(key.R2, key.N), "R^2 mod N below N", nbits, b, kk);
    for (uint32_t j = 0; j < b; j++) {
      const uint64_t Rj = pow2mod(32ull * s, r[j]);
      expect(mod64(key.R2, r[j]) == mulmod(Rj, Rj, r[j]), "R^2 mod N, modulo each prime", nbits, b, kk);
      const uint64_t Rh = pow2mod(32ull * h, r[j]);
      expect(mod64(key.R2h[j], r[j]) == mulmod(Rh, Rh, r[j]) && as64(key.R2h[j]) < r[j], "R_h^2 mod r_i", nbits,
             b, kk);
      expect(mod64(key.R3h[j], r[j]) == mulmod(mulmod(Rh, Rh, r[j]), Rh, r[j]) && as64(key.R3h[j]) < r[j],
             "R_h^3 mod r_i", nbits, b, kk);
      expect((uint32_t)(key.n0h[j] * key.pr[j][0]) == 0xFFFFFFFFu, "-r_i^-1 mod 2^32", nbits, b, kk);
      const uint64_t dj = as64(key.dpr[j]);
      expect(dj < r[j] - 1 && mulmod(e % (r[j] - 1), dj, r[j] - 1) == 1, "e (d mod (r_i - 1)) = 1", nbits, b, kk);
    }
    // Garner coefficients
    expect(mulmod(as64(key.coef[0]), r[1] % r[0], r[0]) == 1, "coef_0 r_1 = 1 mod r_0", nbits, b, kk);
    expect(as64(key.coef[1]) == 0, "coef_1 = 0", nbits, b, kk);
    for (uint32_t i = 2; i < b; i++) {
      uint64_t p = 1;
      for (uint32_t j = 0; j < i; j++) p = mulmod(p, r[j] % r[i], r[i]);
      expect(mulmod(as64(key.coef[i]), p, r[i]) == 1, "coef_i (r_0 ... r_{i-1}) = 1 mod r_i", nbits, b, kk);
    }
    // recombination rows c_i R mod N
    for (uint32_t i = 0; i < b; i++) {
      expect(less(key.crt_sum[i], key.N), "c_i R mod N below N", nbits, b, kk);
      for (uint32_t j = 0; j < b; j++) {
        const uint64_t want = i == j ? pow2mod(32ull * s, r[j]) : 0;
        expect(mod64(key.crt_sum[i], r[j]) == want, "c_i R = delta_ij R modulo r_j", nbits, b, kk);
      }
    }
  }
}

}  // namespace

int main() {
  check_keys(6, 128, 2, 65537, 0x50444D4B4B430001ull);
  check_keys(6, 256, 4, 65537, 0x50444D4B4B430002ull);
  check_keys(3, 128, 2, 3, 0x50444D4B4B430003ull);
  check_keys(3, 256, 4, 17, 0x50444D4B4B430004ull);
  std::printf("%d checks, %d failures\n", g_checks, g_failures);
  return g_failures ? 1 : 0;
}
