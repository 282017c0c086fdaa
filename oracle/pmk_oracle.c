/*
 * PMKRSA oracle — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU restatement of what the PMKRSA hot
 * path computes ("A Variant RSA Acceleration with Parallelization",
 * arXiv 2111.11924).  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference arm may load it.  It shares no code with the
 * product library: its own schoolbook bignum on 32-bit limbs, division by
 * Knuth's Algorithm D (TAOCP Vol. 2, 4.3.1), no Montgomery arithmetic.
 *
 * Functions and the passages they follow:
 *   oracle_modexp      Algorithm 2 (multiply-and-square, bits e_0..e_{l-1}
 *                      scanned upward, final multiply supplies e_l = 1).
 *   oracle_crt         Section 2.1, CRT-RSA equation, read as Garner:
 *                      m_p = c^dp mod p, m_q = c^dq mod q,
 *                      h = qinv (m_p - m_q) mod p, m = m_q + h q.
 *   oracle_keygen      Section 1.1 key initialisation and Algorithm 1
 *                      "Initialization": p != q of n/2 bits, N = pq,
 *                      phi = (p-1)(q-1), d = e^-1 mod phi (extended Euclid).
 *   oracle_keygen_mp   Section 2.1, multi-prime RSA: b distinct primes of
 *                      n/b bits, N their product, phi = prod (r_i - 1).
 *   oracle_crt_mp      multi-prime CRT decryption: the CRT-RSA equation for
 *                      the first two primes, extended one prime at a time
 *                      (Garner's mixed-radix recombination).
 *   oracle_*_chunks    Algorithm 1 "Encryption"/"Decryption" loops: chunk t
 *                      is bound to key t mod K (row-per-key reshape, Sec. 3.1).
 *   oracle_blind_*     Algorithm 1 with the random matrix R (Sec. 3.1):
 *                      encrypt c = m^e, c* = c r^e, c_r = r^e (mod N);
 *                      decrypt r' = c_r^d, m* = c*^d, m' = m* r'^-1 (mod N).
 *
 * Readings where the paper is silent or garbled (kept identical on the
 * product side, which implements them independently):
 *   - random source: SplitMix64 (Steele, Lea, Flood 2014) instead of
 *     /dev/random; key k draws from its own stream, seeded with the k-th
 *     output of a master SplitMix64 stream seeded by the caller, so the K
 *     keys can be generated in parallel as Section 3.3 does with OpenMP;
 *   - primes have exactly n/2 bits with the two top bits set (so N has
 *     exactly n bits), bit 0 set; candidates are rejected by trial division
 *     by the odd primes below 2000, then unless gcd(e, cand-1) = 1, then by
 *     40 Miller-Rabin rounds whose bases are (splitmix64() >> 1) + 2;
 *   - q is redrawn while q == p.
 *
 * Error convention: 0 on success, negative on invalid arguments.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint32_t limb_t;
typedef uint64_t dlimb_t;

/* ------------------------------------------------------------------ */
/* schoolbook bignum: little-endian arrays of 32-bit limbs             */
/* ------------------------------------------------------------------ */

static int bn_len(const limb_t *a, int n) {
  while (n > 0 && a[n - 1] == 0) n--;
  return n;
}

static int bn_cmp(const limb_t *a, int na, const limb_t *b, int nb) {
  na = bn_len(a, na);
  nb = bn_len(b, nb);
  if (na != nb) return na < nb ? -1 : 1;
  for (int i = na - 1; i >= 0; i--)
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  return 0;
}

static void bn_zero(limb_t *a, int n) { memset(a, 0, (size_t)n * sizeof(limb_t)); }

static void bn_copy(limb_t *dst, int nd, const limb_t *src, int ns) {
  for (int i = 0; i < nd; i++) dst[i] = i < ns ? src[i] : 0;
}

/* r[0..n) = a + b (n limbs each), returns carry out */
static limb_t bn_add_n(limb_t *r, const limb_t *a, const limb_t *b, int n) {
  dlimb_t c = 0;
  for (int i = 0; i < n; i++) {
    c += (dlimb_t)a[i] + b[i];
    r[i] = (limb_t)c;
    c >>= 32;
  }
  return (limb_t)c;
}

/* r[0..n) = a - b (n limbs each), returns borrow out */
static limb_t bn_sub_n(limb_t *r, const limb_t *a, const limb_t *b, int n) {
  limb_t borrow = 0;
  for (int i = 0; i < n; i++) {
    dlimb_t d = (dlimb_t)a[i] - b[i] - borrow;
    r[i] = (limb_t)d;
    borrow = (limb_t)((d >> 63) & 1);
  }
  return borrow;
}

/* out[0..na+nb) = a * b  (schoolbook, one row per limb of b) */
static void bn_mul(const limb_t *a, int na, const limb_t *b, int nb, limb_t *out) {
  bn_zero(out, na + nb);
  for (int j = 0; j < nb; j++) {
    dlimb_t carry = 0;
    for (int i = 0; i < na; i++) {
      dlimb_t t = (dlimb_t)a[i] * b[j] + out[i + j] + carry;
      out[i + j] = (limb_t)t;
      carry = t >> 32;
    }
    out[na + j] = (limb_t)carry;
  }
}

static int clz32(limb_t x) {
  int n = 0;
  if (x == 0) return 32;
  while (!(x & 0x80000000u)) { x <<= 1; n++; }
  return n;
}

/*
 * Division with remainder, Knuth Algorithm D (TAOCP Vol. 2, 4.3.1):
 *   u = q v + r, 0 <= r < v.
 * q gets nu - nv + 1 limbs (may be NULL), r gets nv limbs (may be NULL).
 * Returns -1 if v == 0.
 */
static int bn_divmod(const limb_t *u, int nu, const limb_t *v, int nv, limb_t *q, int nq, limb_t *r, int nr) {
  int n = bn_len(v, nv);
  int m = bn_len(u, nu);
  if (n == 0) return -1;
  if (q) bn_zero(q, nq);
  if (m < n) {
    if (r) bn_copy(r, nr, u, m);
    return 0;
  }
  if (n == 1) { /* short division by a single limb */
    dlimb_t rem = 0;
    for (int i = m - 1; i >= 0; i--) {
      dlimb_t cur = (rem << 32) | u[i];
      if (q && i < nq) q[i] = (limb_t)(cur / v[0]);
      rem = cur % v[0];
    }
    if (r) { bn_zero(r, nr); if (nr > 0) r[0] = (limb_t)rem; }
    return 0;
  }
  /* D1: normalise so the divisor's top limb has its top bit set */
  int s = clz32(v[n - 1]);
  limb_t *vn = (limb_t *)malloc(sizeof(limb_t) * (size_t)n);
  limb_t *un = (limb_t *)malloc(sizeof(limb_t) * (size_t)(m + 1));
  for (int i = n - 1; i > 0; i--) vn[i] = s ? (v[i] << s) | (v[i - 1] >> (32 - s)) : v[i];
  vn[0] = v[0] << s;
  un[m] = s ? u[m - 1] >> (32 - s) : 0;
  for (int i = m - 1; i > 0; i--) un[i] = s ? (u[i] << s) | (u[i - 1] >> (32 - s)) : u[i];
  un[0] = u[0] << s;
  const dlimb_t B = (dlimb_t)1 << 32;
  /* D2..D7: one quotient limb per step, from the top */
  for (int j = m - n; j >= 0; j--) {
    /* D3: estimate qhat from the top two limbs of the current remainder */
    dlimb_t num = ((dlimb_t)un[j + n] << 32) | un[j + n - 1];
    dlimb_t qhat = num / vn[n - 1];
    dlimb_t rhat = num % vn[n - 1];
    while (qhat >= B || qhat * vn[n - 2] > ((rhat << 32) | un[j + n - 2])) {
      qhat--;
      rhat += vn[n - 1];
      if (rhat >= B) break;
    }
    /* D4: multiply and subtract qhat * vn from un[j .. j+n] */
    dlimb_t carry = 0;
    limb_t borrow = 0;
    for (int i = 0; i < n; i++) {
      dlimb_t p = qhat * vn[i] + carry;
      carry = p >> 32;
      dlimb_t d = (dlimb_t)un[i + j] - (limb_t)p - borrow;
      un[i + j] = (limb_t)d;
      borrow = (limb_t)((d >> 63) & 1);
    }
    dlimb_t d = (dlimb_t)un[j + n] - carry - borrow;
    un[j + n] = (limb_t)d;
    /* D5/D6: the estimate was one too large: add the divisor back */
    if ((d >> 63) & 1) {
      qhat--;
      dlimb_t c = 0;
      for (int i = 0; i < n; i++) {
        c += (dlimb_t)un[i + j] + vn[i];
        un[i + j] = (limb_t)c;
        c >>= 32;
      }
      un[j + n] = (limb_t)(un[j + n] + c);
    }
    if (q && j < nq) q[j] = (limb_t)qhat;
  }
  /* D8: unnormalise the remainder */
  if (r) {
    bn_zero(r, nr);
    for (int i = 0; i < n && i < nr; i++) r[i] = s ? (un[i] >> s) | (un[i + 1] << (32 - s)) : un[i];
  }
  free(vn);
  free(un);
  return 0;
}

/* out[0..n) = (a * b) mod N, with a, b of n limbs */
static void bn_mulmod(const limb_t *a, const limb_t *b, const limb_t *N, int n, limb_t *out) {
  limb_t *t = (limb_t *)malloc(sizeof(limb_t) * (size_t)(2 * n));
  bn_mul(a, n, b, n, t);
  bn_divmod(t, 2 * n, N, n, NULL, 0, out, n);
  free(t);
}

static int bn_bit(const limb_t *e, int i) { return (int)((e[i >> 5] >> (i & 31)) & 1u); }

/*
 * Algorithm 2, multiply-and-square exponentiation (base 2):
 *   y = 1, x = x mod N
 *   for i in [0, l): if e_i = 1 then y = y x mod N;  x = x x mod N
 *   return y x mod N
 * where e = (e_l ... e_0)_2 with e_l = 1 its top set bit.  e = 0 and N < 2
 * are rejected (the final multiply assumes e_l = 1).
 */
static int modexp(const limb_t *x, int nx, const limb_t *e, int ne, const limb_t *N, int n, limb_t *out) {
  ne = bn_len(e, ne);
  if (ne == 0) return -1;
  if (bn_len(N, n) == 0 || (bn_len(N, n) == 1 && N[0] < 2)) return -1;
  int l = 32 * (ne - 1) + (31 - clz32(e[ne - 1]));
  limb_t *y = (limb_t *)calloc((size_t)n, sizeof(limb_t));
  limb_t *xx = (limb_t *)calloc((size_t)n, sizeof(limb_t));
  y[0] = 1;
  bn_divmod(x, nx, N, n, NULL, 0, xx, n);
  for (int i = 0; i < l; i++) {
    if (bn_bit(e, i)) bn_mulmod(y, xx, N, n, y);
    bn_mulmod(xx, xx, N, n, xx);
  }
  bn_mulmod(y, xx, N, n, out);
  free(y);
  free(xx);
  return 0;
}

/*
 * Garner form of the CRT-RSA decryption (Section 2.1):
 *   m_p = c^dp mod p,  m_q = c^dq mod q,
 *   h = qinv (m_p - m_q) mod p,  m = m_q + h q.
 * p, q, dp, dq, qinv have h limbs; c and out have 2h limbs.
 */
static int crt(const limb_t *c, const limb_t *dp, const limb_t *dq, const limb_t *p, const limb_t *q,
               const limb_t *qinv, int h, limb_t *out) {
  int n = 2 * h;
  limb_t *mp = (limb_t *)calloc((size_t)h, sizeof(limb_t));
  limb_t *mq = (limb_t *)calloc((size_t)h, sizeof(limb_t));
  limb_t *mqp = (limb_t *)calloc((size_t)h, sizeof(limb_t));
  limb_t *diff = (limb_t *)calloc((size_t)h, sizeof(limb_t));
  limb_t *hh = (limb_t *)calloc((size_t)h, sizeof(limb_t));
  limb_t *hq = (limb_t *)calloc((size_t)n, sizeof(limb_t));
  int rc = modexp(c, n, dp, h, p, h, mp);
  if (!rc) rc = modexp(c, n, dq, h, q, h, mq);
  if (!rc) {
    bn_divmod(mq, h, p, h, NULL, 0, mqp, h);           /* m_q mod p */
    if (bn_cmp(mp, h, mqp, h) >= 0) {
      bn_sub_n(diff, mp, mqp, h);
    } else {                                             /* m_p - m_q + p */
      bn_sub_n(diff, p, mqp, h);
      bn_add_n(diff, diff, mp, h);
    }
    bn_mulmod(diff, qinv, p, h, hh);                     /* h = qinv (m_p - m_q) mod p */
    bn_mul(hh, h, q, h, hq);                             /* h q */
    limb_t *mq2 = (limb_t *)calloc((size_t)n, sizeof(limb_t));
    bn_copy(mq2, n, mq, h);
    bn_add_n(out, hq, mq2, n);                           /* m = m_q + h q  (< N, no carry) */
    free(mq2);
  }
  free(mp); free(mq); free(mqp); free(diff); free(hh); free(hq);
  return rc;
}

/* ------------------------------------------------------------------ */
/* signed bignum pieces for the extended Euclidean algorithm           */
/* ------------------------------------------------------------------ */

/*
 * inv = a^-1 mod m by the extended Euclidean algorithm, tracking the
 * coefficient of a with an explicit sign.  All arrays have n limbs.
 * Returns 0 on success, -1 if gcd(a, m) != 1.
 */
static int bn_modinv(const limb_t *a, const limb_t *m, int n, limb_t *inv) {
  int w = 2 * n + 2;
  limb_t *r0 = calloc((size_t)w, 4), *r1 = calloc((size_t)w, 4), *rr = calloc((size_t)w, 4);
  limb_t *qq = calloc((size_t)w, 4), *prod = calloc((size_t)(2 * w), 4);
  limb_t *t0 = calloc((size_t)w, 4), *t1 = calloc((size_t)w, 4), *tn = calloc((size_t)w, 4);
  int s0 = 0, s1 = 0, sn = 0; /* sign flags: 1 = negative */
  int rc = -1;
  bn_copy(r0, w, m, n);
  bn_divmod(a, n, m, n, NULL, 0, r1, w); /* r1 = a mod m */
  t1[0] = 1;                              /* t0 = 0, t1 = 1 */
  while (bn_len(r1, w) > 0) {
    bn_divmod(r0, w, r1, w, qq, w, rr, w);  /* r0 = qq r1 + rr */
    /* t_new = t0 - qq * t1 */
    bn_mul(qq, w, t1, w, prod);
    int sp = s1;                            /* sign of qq * t1 */
    limb_t *pm = prod;                      /* magnitude fits in w limbs */
    if (sp == s0) {                         /* t0 - p, same signs: subtract magnitudes */
      if (bn_cmp(t0, w, pm, w) >= 0) { bn_sub_n(tn, t0, pm, w); sn = s0; }
      else { bn_sub_n(tn, pm, t0, w); sn = !s0; }
    } else {                                /* opposite signs: add magnitudes, keep t0's sign */
      bn_add_n(tn, t0, pm, w);
      sn = s0;
    }
    if (bn_len(tn, w) == 0) sn = 0;
    memcpy(r0, r1, (size_t)w * 4);
    memcpy(r1, rr, (size_t)w * 4);
    memcpy(t0, t1, (size_t)w * 4); s0 = s1;
    memcpy(t1, tn, (size_t)w * 4); s1 = sn;
  }
  if (bn_len(r0, w) == 1 && r0[0] == 1) {
    limb_t *mw = calloc((size_t)w, 4);
    bn_copy(mw, w, m, n);
    bn_divmod(t0, w, mw, w, NULL, 0, rr, w);   /* |t0| mod m */
    if (s0 && bn_len(rr, w) > 0) bn_sub_n(rr, mw, rr, w);
    bn_copy(inv, n, rr, w);
    free(mw);
    rc = 0;
  }
  free(r0); free(r1); free(rr); free(qq); free(prod); free(t0); free(t1); free(tn);
  return rc;
}

/* ------------------------------------------------------------------ */
/* key generation                                                      */
/* ------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): one output per call. */
static uint64_t splitmix64(uint64_t *state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static uint64_t gcd_u64(uint64_t a, uint64_t b) {
  while (b) { uint64_t t = a % b; a = b; b = t; }
  return a;
}

/* one Miller-Rabin round to base `base` (< n), by plain Algorithm 2 modexp */
static int mr_round(const limb_t *n, int h, uint64_t base) {
  limb_t *n1 = calloc((size_t)h, 4), *dd = calloc((size_t)h, 4), *x = calloc((size_t)h, 4);
  limb_t *b = calloc((size_t)h, 4), *one = calloc((size_t)h, 4);
  one[0] = 1;
  bn_sub_n(n1, n, one, h);                  /* n - 1 */
  int s = 0;
  while (!bn_bit(n1, s)) s++;
  for (int i = 0; i < h; i++) {             /* dd = (n - 1) >> s */
    int bit = s + 32 * i;
    limb_t lo = (bit >> 5) < h ? n1[bit >> 5] >> (bit & 31) : 0;
    limb_t hi = ((bit >> 5) + 1 < h && (bit & 31)) ? n1[(bit >> 5) + 1] << (32 - (bit & 31)) : 0;
    dd[i] = lo | hi;
  }
  b[0] = (limb_t)base;
  if (h > 1) b[1] = (limb_t)(base >> 32);
  modexp(b, h, dd, h, n, h, x);
  int pass = 0;
  if (bn_cmp(x, h, one, h) == 0 || bn_cmp(x, h, n1, h) == 0) pass = 1;
  for (int i = 1; i < s && !pass; i++) {
    bn_mulmod(x, x, n, h, x);
    if (bn_cmp(x, h, n1, h) == 0) pass = 1;
    else if (bn_cmp(x, h, one, h) == 0) break;
  }
  free(n1); free(dd); free(x); free(b); free(one);
  return pass;
}

/*
 * draw a prime of exactly `bits` bits (bits a multiple of 64) into p[0..bits/32),
 * whose top byte is at least min_top (>= 192: the top two bits are always set)
 */
static void gen_prime(uint64_t *rng, int bits, uint64_t e, const int *small, int nsmall, int min_top, limb_t *p) {
  int h = bits / 32;
  limb_t *em1 = calloc((size_t)h, 4), *one = calloc((size_t)h, 4);
  limb_t ev[2] = {(limb_t)e, (limb_t)(e >> 32)};
  limb_t rem[2];
  one[0] = 1;
  for (;;) {
    for (int w = 0; w < bits / 64; w++) {
      uint64_t r = splitmix64(rng);
      p[2 * w] = (limb_t)r;
      p[2 * w + 1] = (limb_t)(r >> 32);
    }
    p[h - 1] |= 0xC0000000u; /* exactly `bits` bits, top two set */
    p[0] |= 1u;
    if ((int)(p[h - 1] >> 24) < min_top) continue;
    int composite = 0;
    for (int i = 0; i < nsmall && !composite; i++) {
      limb_t sp = (limb_t)small[i], r1[1];
      bn_divmod(p, h, &sp, 1, NULL, 0, r1, 1);
      if (r1[0] == 0) composite = 1;
    }
    if (composite) continue;
    bn_sub_n(em1, p, one, h);
    bn_divmod(em1, h, ev, 2, NULL, 0, rem, 2);
    uint64_t rm = (uint64_t)rem[0] | ((uint64_t)rem[1] << 32);
    if (gcd_u64(e, rm) != 1) continue;
    int ok = 1;
    for (int round = 0; round < 40 && ok; round++) {
      uint64_t base = (splitmix64(rng) >> 1) + 2;
      ok = mr_round(p, h, base);
    }
    if (ok) break;
  }
  free(em1);
  free(one);
}

/* the odd primes below 2000, by trial division; returns their count */
static int small_primes(int *small) {
  int nsmall = 0;
  for (int c = 3; c < 2000; c += 2) {
    int pr = 1;
    for (int f = 3; f * f <= c; f += 2)
      if (c % f == 0) { pr = 0; break; }
    if (pr) small[nsmall++] = c;
  }
  return nsmall;
}

/*
 * The least top byte T (at least 192) with T^b >= 2^(8b - 1): b primes of k
 * bits whose top bytes are all >= T have a product of at least
 * (T / 256)^b 2^(bk) >= 2^(bk - 1), so the modulus has exactly bk bits.
 */
static int mp_top_floor(int b) {
  const uint64_t need = 1ull << (8 * b - 1);
  int t = 1;
  for (;; t++) {
    uint64_t v = 1;
    for (int i = 0; i < b; i++) v *= (uint64_t)t;
    if (v >= need) break;
  }
  return t < 192 ? 192 : t;
}

/*
 * Multi-prime CRT decryption of one chunk (Section 2.1, multi-prime RSA),
 * b primes r_0 .. r_{b-1} of h limbs each, c and out of b h limbs:
 *   m_i = c^{d_i} mod r_i  (d_i = d mod (r_i - 1));
 *   the first recombination is the CRT-RSA equation with p = r_0, q = r_1:
 *     x = coef_0 (m_0 - m_1) mod r_0  (coef_0 = r_1^-1 mod r_0),  m = m_1 + x r_1;
 *   each further prime r_i extends it the same way over the product
 *   P_i = r_0 ... r_{i-1} of the primes already combined:
 *     x = coef_i (m_i - m) mod r_i  (coef_i = P_i^-1 mod r_i),  m = m + x P_i.
 * m stays below the product of the primes combined so far (Garner's
 * mixed-radix form); after the last prime it is c^d mod N.
 */
static int crt_mp(const limb_t *c, int b, int h, const limb_t *r, const limb_t *dexp, const limb_t *coef,
                  limb_t *out) {
  const int s = b * h;
  limb_t *mi = calloc((size_t)s, 4), *m = calloc((size_t)s, 4), *P = calloc((size_t)s, 4);
  limb_t *x = calloc((size_t)h, 4), *diff = calloc((size_t)h, 4), *xr = calloc((size_t)(s + h), 4);
  limb_t *tmp = calloc((size_t)(s + h), 4);
  int rc = 0;
  for (int i = 0; i < b && !rc; i++) rc = modexp(c, s, dexp + (size_t)i * h, h, r + (size_t)i * h, h, mi + (size_t)i * h);
  if (!rc) {
    /* the running value starts at m_1, its product at r_1; then r_0, r_2, r_3, ... */
    bn_copy(m, s, mi + h, h);
    bn_copy(P, s, r + h, h);
    int len = h;
    for (int step = 0; step < b - 1; step++) {
      const int i = step == 0 ? 0 : step + 1;
      const limb_t *ri = r + (size_t)i * h, *m_i = mi + (size_t)i * h;
      bn_divmod(m, len, ri, h, NULL, 0, x, h);           /* m mod r_i */
      if (bn_cmp(m_i, h, x, h) >= 0) {
        bn_sub_n(diff, m_i, x, h);
      } else {                                           /* m_i - m + r_i */
        bn_sub_n(diff, ri, x, h);
        bn_add_n(diff, diff, m_i, h);
      }
      bn_mulmod(diff, coef + (size_t)i * h, ri, h, x);   /* x = coef_i (m_i - m) mod r_i */
      bn_mul(P, len, x, h, xr);                          /* x P_i */
      bn_copy(tmp, len + h, m, len);
      bn_add_n(m, tmp, xr, len + h);                     /* m + x P_i  (< P_i r_i, no carry) */
      bn_mul(P, len, ri, h, tmp);                        /* P_{i+1} = P_i r_i */
      bn_copy(P, s, tmp, len + h);
      len += h;
    }
    bn_copy(out, s, m, s);
  }
  free(mi); free(m); free(P); free(x); free(diff); free(xr); free(tmp);
  return rc;
}

/* ------------------------------------------------------------------ */
/* exported entry points                                               */
/* ------------------------------------------------------------------ */

int oracle_mulmod(const uint32_t *a, const uint32_t *b, const uint32_t *N, int n, uint32_t *out) {
  if (n <= 0 || bn_len(N, n) == 0) return -1;
  bn_mulmod(a, b, N, n, out);
  return 0;
}

int oracle_divmod(const uint32_t *u, int nu, const uint32_t *v, int nv, uint32_t *q, int nq, uint32_t *r, int nr) {
  return bn_divmod(u, nu, v, nv, q, nq, r, nr);
}

int oracle_modexp(const uint32_t *x, int nx, const uint32_t *e, int ne, const uint32_t *N, int n, uint32_t *out) {
  return modexp(x, nx, e, ne, N, n, out);
}

int oracle_crt(const uint32_t *c, const uint32_t *dp, const uint32_t *dq, const uint32_t *p, const uint32_t *q,
               const uint32_t *qinv, int h, uint32_t *out) {
  return crt(c, dp, dq, p, q, qinv, h, out);
}

int oracle_modinv(const uint32_t *a, const uint32_t *m, int n, uint32_t *inv) {
  return bn_modinv(a, m, n, inv);
}

/*
 * K key pairs of nbits (a multiple of 128, >= 128) with public exponent e
 * (odd, >= 3).  Output arrays, key-major:
 *   N, d: K x nbits/32 limbs;  p, q, dp, dq, qinv: K x nbits/64 limbs.
 */
int oracle_keygen(uint32_t K, uint32_t nbits, uint64_t e, uint64_t seed, uint32_t *N, uint32_t *d,
                  uint32_t *p, uint32_t *q, uint32_t *dp, uint32_t *dq, uint32_t *qinv) {
  if (K == 0 || nbits < 128 || nbits % 128 != 0 || e < 3 || !(e & 1)) return -1;
  int s = (int)nbits / 32, h = s / 2;
  int small[400];
  int nsmall = small_primes(small);
  uint64_t master = seed;
  limb_t *one = calloc((size_t)h, 4), *pm1 = calloc((size_t)h, 4), *qm1 = calloc((size_t)h, 4);
  limb_t *phi = calloc((size_t)s, 4), *ew = calloc((size_t)s, 4);
  one[0] = 1;
  ew[0] = (limb_t)e;
  ew[1] = (limb_t)(e >> 32);
  for (uint32_t k = 0; k < K; k++) {
    limb_t *pk = p + (size_t)k * h, *qk = q + (size_t)k * h;
    uint64_t rng = splitmix64(&master);   /* this key's own stream */
    gen_prime(&rng, (int)nbits / 2, e, small, nsmall, 192, pk);
    do {
      gen_prime(&rng, (int)nbits / 2, e, small, nsmall, 192, qk);
    } while (bn_cmp(pk, h, qk, h) == 0);
    bn_mul(pk, h, qk, h, N + (size_t)k * s);                 /* N = p q */
    bn_sub_n(pm1, pk, one, h);
    bn_sub_n(qm1, qk, one, h);
    bn_mul(pm1, h, qm1, h, phi);                              /* phi = (p-1)(q-1) */
    if (bn_modinv(ew, phi, s, d + (size_t)k * s)) return -2;  /* d = e^-1 mod phi */
    bn_divmod(d + (size_t)k * s, s, pm1, h, NULL, 0, dp + (size_t)k * h, h);  /* dp = d mod (p-1) */
    bn_divmod(d + (size_t)k * s, s, qm1, h, NULL, 0, dq + (size_t)k * h, h);  /* dq = d mod (q-1) */
    if (bn_modinv(qk, pk, h, qinv + (size_t)k * h)) return -2;                /* qinv = q^-1 mod p */
  }
  free(one); free(pm1); free(qm1); free(phi); free(ew);
  return 0;
}

/*
 * Algorithm 1 loops over a range of chunks: out_t = in_t ^ exp_{t mod K} mod N_{t mod K}
 * for t in [t0, t1).  in/out: chunk-major, s limbs per chunk.  exps: K x ne limbs.
 */
int oracle_modexp_chunks(const uint32_t *in, uint32_t *out, int s, const uint32_t *exps, int ne,
                         const uint32_t *mods, int K, long t0, long t1) {
  for (long t = t0; t < t1; t++) {
    int k = (int)(t % K);
    int rc = modexp(in + (size_t)t * s, s, exps + (size_t)k * ne, ne, mods + (size_t)k * s, s, out + (size_t)t * s);
    if (rc) return rc;
  }
  return 0;
}

/* CRT decryption of chunks [t0, t1); key arrays are K x s/2 limbs each. */
int oracle_crt_chunks(const uint32_t *in, uint32_t *out, int s, const uint32_t *dp, const uint32_t *dq,
                      const uint32_t *p, const uint32_t *q, const uint32_t *qinv, int K, long t0, long t1) {
  int h = s / 2;
  for (long t = t0; t < t1; t++) {
    size_t k = (size_t)(t % K);
    int rc = crt(in + (size_t)t * s, dp + k * h, dq + k * h, p + k * h, q + k * h, qinv + k * h, h, out + (size_t)t * s);
    if (rc) return rc;
  }
  return 0;
}

/*
 * Multi-prime key pairs (Section 2.1, multi-prime RSA): K keys of nbits with
 * b in [2, 4] distinct primes of nbits / b bits each (nbits a multiple of 128
 * and of 64 b).  Key k draws r_0, r_1, ... in order from its own stream as in
 * oracle_keygen; every prime's top byte is at least mp_top_floor(b), so N
 * has exactly nbits bits, and r_i is redrawn while it equals an earlier prime.
 * For b = 2 this is oracle_keygen's key (p = r_0, q = r_1).  Outputs, key-major:
 *   N, d: K x nbits/32 limbs;  primes, dexp, coef: K x b x nbits/(32 b) limbs,
 *   dexp_i = d mod (r_i - 1), coef_0 = r_1^-1 mod r_0, coef_1 = 0,
 *   coef_i = (r_0 ... r_{i-1})^-1 mod r_i for i >= 2.
 */
int oracle_keygen_mp(uint32_t K, uint32_t nbits, uint32_t b, uint64_t e, uint64_t seed, uint32_t *N, uint32_t *d,
                     uint32_t *primes, uint32_t *dexp, uint32_t *coef) {
  if (K == 0 || b < 2 || b > 4 || nbits < 128 || nbits % 128 || nbits % (64 * b) || e < 3 || !(e & 1)) return -1;
  const int s = (int)nbits / 32, h = s / (int)b, top = mp_top_floor((int)b);
  int small[400];
  int nsmall = small_primes(small);
  uint64_t master = seed;
  limb_t *phi = calloc((size_t)s, 4), *ew = calloc((size_t)s, 4), *acc = calloc((size_t)s, 4);
  limb_t *tmp = calloc((size_t)s, 4), *rm1 = calloc((size_t)h, 4), *one = calloc((size_t)h, 4);
  limb_t *x = calloc((size_t)h, 4);
  int rc = 0;
  one[0] = 1;
  ew[0] = (limb_t)e;
  ew[1] = (limb_t)(e >> 32);
  for (uint32_t k = 0; k < K && !rc; k++) {
    limb_t *r = primes + (size_t)k * s, *Nk = N + (size_t)k * s, *dk = d + (size_t)k * s;
    uint64_t rng = splitmix64(&master);
    for (uint32_t i = 0; i < b; i++) {
      int dup;
      do {
        gen_prime(&rng, (int)nbits / (int)b, e, small, nsmall, top, r + (size_t)i * h);
        dup = 0;
        for (uint32_t j = 0; j < i; j++)
          if (bn_cmp(r + (size_t)j * h, h, r + (size_t)i * h, h) == 0) dup = 1;
      } while (dup);
    }
    /* N = r_0 ... r_{b-1},  phi = (r_0 - 1) ... (r_{b-1} - 1) */
    bn_copy(Nk, s, r, h);
    bn_sub_n(rm1, r, one, h);
    bn_copy(phi, s, rm1, h);
    for (uint32_t i = 1; i < b; i++) {
      bn_mul(Nk, (int)i * h, r + (size_t)i * h, h, tmp);
      bn_copy(Nk, s, tmp, (int)(i + 1) * h);
      bn_sub_n(rm1, r + (size_t)i * h, one, h);
      bn_mul(phi, (int)i * h, rm1, h, tmp);
      bn_copy(phi, s, tmp, (int)(i + 1) * h);
    }
    if (bn_modinv(ew, phi, s, dk)) { rc = -2; break; }           /* d = e^-1 mod phi */
    for (uint32_t i = 0; i < b; i++) {
      bn_sub_n(rm1, r + (size_t)i * h, one, h);
      bn_divmod(dk, s, rm1, h, NULL, 0, dexp + (size_t)k * s + (size_t)i * h, h);  /* d mod (r_i - 1) */
    }
    limb_t *ck = coef + (size_t)k * s;
    bn_zero(ck, s);
    if (bn_modinv(r + h, r, h, ck)) { rc = -2; break; }          /* r_1^-1 mod r_0 */
    bn_copy(acc, s, r, h);                                        /* acc = r_0 r_1 ... r_{i-1} */
    for (uint32_t i = 1; i < b; i++) {
      if (i >= 2) {
        bn_divmod(acc, (int)i * h, r + (size_t)i * h, h, NULL, 0, x, h);
        if (bn_modinv(x, r + (size_t)i * h, h, ck + (size_t)i * h)) { rc = -2; break; }
      }
      bn_mul(acc, (int)i * h, r + (size_t)i * h, h, tmp);
      bn_copy(acc, s, tmp, (int)(i + 1) * h);
    }
  }
  free(phi); free(ew); free(acc); free(tmp); free(rm1); free(one); free(x);
  return rc;
}

/* multi-prime CRT decryption of one value: b primes of h limbs, c and out of b h limbs */
int oracle_crt_mp(const uint32_t *c, int b, int h, const uint32_t *primes, const uint32_t *dexp, const uint32_t *coef,
                  uint32_t *out) {
  if (b < 2 || h <= 0) return -1;
  return crt_mp(c, b, h, primes, dexp, coef, out);
}

/* multi-prime CRT decryption of chunks [t0, t1), key t mod K; key arrays K x b h limbs */
int oracle_crt_mp_chunks(const uint32_t *in, uint32_t *out, int s, int b, const uint32_t *primes,
                         const uint32_t *dexp, const uint32_t *coef, int K, long t0, long t1) {
  if (b < 2 || s % b) return -1;
  const int h = s / b;
  for (long t = t0; t < t1; t++) {
    size_t k = (size_t)(t % K);
    int rc = crt_mp(in + (size_t)t * s, b, h, primes + k * s, dexp + k * s, coef + k * s, out + (size_t)t * s);
    if (rc) return rc;
  }
  return 0;
}

/*
 * Algorithm 1 with blinding, chunks [t0, t1), key t mod K (s-limb values):
 *   encrypt:  c_t = m_t^e,  c*_t = c_t r_t^e,  c_r,t = r_t^e   (mod N_k)
 */
int oracle_blind_encrypt_chunks(const uint32_t *m, const uint32_t *rnd, uint32_t *cstar, uint32_t *cr, int s,
                                const uint32_t *e, int ne, const uint32_t *mods, int K, long t0, long t1) {
  limb_t *c = (limb_t *)calloc((size_t)s, sizeof(limb_t));
  int rc = 0;
  for (long t = t0; t < t1 && !rc; t++) {
    const limb_t *N = mods + (size_t)(t % K) * s;
    rc = modexp(m + (size_t)t * s, s, e, ne, N, s, c);                          /* c = m^e */
    if (!rc) rc = modexp(rnd + (size_t)t * s, s, e, ne, N, s, cr + (size_t)t * s); /* c_r = r^e */
    if (!rc) bn_mulmod(c, cr + (size_t)t * s, N, s, cstar + (size_t)t * s);       /* c* = c r^e */
  }
  free(c);
  return rc;
}

/*
 *   decrypt:  r' = c_r^d,  m* = c*^d,  m' = m* r'^-1   (mod N_k)
 * Returns -3 if some r' has no inverse modulo N_k.
 */
int oracle_blind_decrypt_chunks(const uint32_t *cstar, const uint32_t *cr, uint32_t *m, int s, const uint32_t *exps,
                                int ne, const uint32_t *mods, int K, long t0, long t1) {
  limb_t *rp = (limb_t *)calloc((size_t)s, sizeof(limb_t));
  limb_t *ms = (limb_t *)calloc((size_t)s, sizeof(limb_t));
  limb_t *ri = (limb_t *)calloc((size_t)s, sizeof(limb_t));
  int rc = 0;
  for (long t = t0; t < t1 && !rc; t++) {
    const limb_t *N = mods + (size_t)(t % K) * s, *d = exps + (size_t)(t % K) * ne;
    rc = modexp(cr + (size_t)t * s, s, d, ne, N, s, rp);                    /* r' = c_r^d */
    if (!rc) rc = modexp(cstar + (size_t)t * s, s, d, ne, N, s, ms);      /* m* = c*^d */
    if (!rc && bn_modinv(rp, N, s, ri)) rc = -3;                           /* r'^-1 */
    if (!rc) bn_mulmod(ms, ri, N, s, m + (size_t)t * s);                   /* m' = m* r'^-1 */
  }
  free(rp); free(ms); free(ri);
  return rc;
}
