// Host check of the exponent schedules the kernels walk (the left-to-right
// sliding-window form of Algorithm 2's square-and-multiply, and the joint
// schedule of the blinded CRT decryption).  Replaying a schedule on plain
// integers must give back its exponent exactly, with every odd-power index
// inside the table bound.  Built with g++ against keygen.cpp; no GPU.
//
// Replay rules:
//   single schedule: steps[0] = idx loads x^(2 idx + 1); each later step
//     (nsq << 8) | idx squares nsq times, then multiplies by x^(2 idx + 1)
//     unless idx = 0xFF.  So the exponent is rebuilt by E = E * 2^nsq, then
//     E += 2 idx + 1.
//   joint schedule: each step (nsq << 16) | (ia << 8) | ib squares nsq times
//     (nsq = 0 on the first step), then multiplies by A^(2 ia + 1) and by
//     B^(2 ib + 1) (0xFF: none), rebuilding both exponents side by side.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "pmk_internal.h"

namespace {

using Big = std::vector<uint32_t>;  // little-endian 32-bit limbs

void shl(Big &x, uint32_t n) {
  const uint32_t words = n / 32, bits = n % 32;
  Big y(x.size() + words + 1, 0);
  for (size_t i = 0; i < x.size(); i++) {
    const uint64_t v = (uint64_t)x[i] << bits;
    y[i + words] |= (uint32_t)v;
    y[i + words + 1] |= (uint32_t)(v >> 32);
  }
  x.swap(y);
}

void add_small(Big &x, uint32_t v) {
  uint64_t c = v;
  for (size_t i = 0; i < x.size() && c; i++) {
    c += x[i];
    x[i] = (uint32_t)c;
    c >>= 32;
  }
  if (c) x.push_back((uint32_t)c);
}

bool same(const Big &x, const uint32_t *e, int nlimbs) {
  for (size_t i = 0; i < x.size(); i++)
    if (x[i] != ((int)i < nlimbs ? e[i] : 0u)) return false;
  for (int i = (int)x.size(); i < nlimbs; i++)
    if (e[i]) return false;
  return true;
}

bool is_zero(const uint32_t *e, int nlimbs) {
  for (int i = 0; i < nlimbs; i++)
    if (e[i]) return false;
  return true;
}

uint64_t g_state = 0x50444D4B5343484Bull;
uint32_t rnd() {  // xorshift64*
  g_state ^= g_state >> 12;
  g_state ^= g_state << 25;
  g_state ^= g_state >> 27;
  return (uint32_t)((g_state * 0x2545F4914F6CDD1Dull) >> 32);
}

int g_failures = 0, g_checks = 0;

void fail(const char *what, int nlimbs, uint32_t w) {
  if (g_failures++ < 10) std::printf("FAIL %s (limbs %d, window %u)\n", what, nlimbs, w);
}

void check_single(const uint32_t *e, int nlimbs, uint32_t w) {
  g_checks++;
  const pmk::Schedule s = pmk::make_schedule(e, nlimbs, w);
  const uint32_t bound = 1u << (w - 1);  // odd powers in the table
  if (is_zero(e, nlimbs)) {
    if (!s.steps.empty()) fail("zero exponent gave steps", nlimbs, w);
    return;
  }
  if (s.steps.empty() || s.steps[0] >= bound) return fail("first step", nlimbs, w);
  Big x(1, 0);
  add_small(x, 2 * s.steps[0] + 1);
  uint32_t seen = s.steps[0];
  for (size_t i = 1; i < s.steps.size(); i++) {
    const uint32_t nsq = s.steps[i] >> 8, idx = s.steps[i] & 0xFFu;
    shl(x, nsq);
    if (idx != 0xFFu) {
      if (idx >= bound) return fail("index beyond the table", nlimbs, w);
      if (nsq == 0) return fail("multiply without a squaring", nlimbs, w);
      seen = idx > seen ? idx : seen;
      add_small(x, 2 * idx + 1);
    }
  }
  if (seen != s.maxidx) fail("maxidx", nlimbs, w);
  if (!same(x, e, nlimbs)) fail("replay differs from the exponent", nlimbs, w);
}

void check_joint(const uint32_t *ea, const uint32_t *eb, int nlimbs) {
  g_checks++;
  const pmk::Schedule2 s = pmk::make_schedule2(ea, eb, nlimbs);
  if (is_zero(ea, nlimbs) || is_zero(eb, nlimbs)) {
    if (!s.steps.empty()) fail("joint: zero exponent gave steps", nlimbs, 4);
    return;
  }
  if (s.steps.empty() || (s.steps[0] >> 16) != 0) return fail("joint: first step", nlimbs, 4);
  if (s.maxa > 7 || s.maxb > 7) return fail("joint: table bound", nlimbs, 4);
  Big xa(1, 0), xb(1, 0);
  uint32_t seen_a = 0, seen_b = 0;
  for (size_t i = 0; i < s.steps.size(); i++) {
    const uint32_t nsq = s.steps[i] >> 16, ia = (s.steps[i] >> 8) & 0xFFu, ib = s.steps[i] & 0xFFu;
    if (i > 0 && nsq == 0) return fail("joint: step without a squaring", nlimbs, 4);
    if (i == 0 && ia == 0xFFu && ib == 0xFFu) return fail("joint: empty first step", nlimbs, 4);
    shl(xa, nsq);
    shl(xb, nsq);
    if (ia != 0xFFu) {
      if (ia > s.maxa) return fail("joint: A index beyond maxa", nlimbs, 4);
      seen_a = ia > seen_a ? ia : seen_a;
      add_small(xa, 2 * ia + 1);
    }
    if (ib != 0xFFu) {
      if (ib > s.maxb) return fail("joint: B index beyond maxb", nlimbs, 4);
      seen_b = ib > seen_b ? ib : seen_b;
      add_small(xb, 2 * ib + 1);
    }
  }
  if (seen_a != s.maxa || seen_b != s.maxb) fail("joint: maxa / maxb", nlimbs, 4);
  if (!same(xa, ea, nlimbs) || !same(xb, eb, nlimbs)) fail("joint: replay differs", nlimbs, 4);
}

// Exponents of nlimbs limbs: random with a random top, sparse, dense, and
// special values (0, 1, 2, 3, 65537, 2^k, 2^k - 1, alternating bits).
std::vector<Big> exponents(int nlimbs) {
  std::vector<Big> v;
  for (int t = 0; t < 12; t++) {
    Big e(nlimbs);
    for (auto &w : e) w = rnd();
    const int top = (int)(rnd() % (32 * nlimbs));  // clear the bits above a random top bit
    for (int b = top + 1; b < 32 * nlimbs; b++) e[b / 32] &= ~(1u << (b % 32));
    v.push_back(e);
  }
  for (int t = 0; t < 4; t++) {  // sparse: a few random bits
    Big e(nlimbs, 0);
    for (int k = 0; k < 5; k++) {
      const int b = (int)(rnd() % (32 * nlimbs));
      e[b / 32] |= 1u << (b % 32);
    }
    v.push_back(e);
  }
  for (uint32_t small : {0u, 1u, 2u, 3u, 65537u}) {
    Big e(nlimbs, 0);
    e[0] = small;
    v.push_back(e);
  }
  Big p2(nlimbs, 0), ones(nlimbs, 0xFFFFFFFFu), alt(nlimbs, 0xAAAAAAAAu), alt5(nlimbs, 0x55555555u);
  p2[nlimbs - 1] = 0x80000000u;
  v.push_back(p2);
  v.push_back(ones);
  v.push_back(alt);
  v.push_back(alt5);
  return v;
}

}  // namespace

int main() {
  for (int nlimbs : {1, 2, 3, 16, 32, 64, 96, 128, 256}) {
    const std::vector<Big> es = exponents(nlimbs);
    for (uint32_t w = 1; w <= pmk::kWindowFull; w++)
      for (const Big &e : es) check_single(e.data(), nlimbs, w);
    for (size_t i = 0; i < es.size(); i++) check_joint(es[i].data(), es[(i * 7 + 3) % es.size()].data(), nlimbs);
  }
  std::printf("%d schedules checked, %d failures\n", g_checks, g_failures);
  return g_failures ? 1 : 0;
}
