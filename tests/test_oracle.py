"""Pins for the CPU oracle: every check compares it with something other than itself.

Sources of truth used here:
  * the textbook 3233 worked example (tests/golden/textbook_rsa_3233.txt);
  * brute force over every message for tiny moduli: the plain definition
    x^e = x * x * ... * x (mod N) as repeated multiplication, and the RSA /
    PMKRSA round trip m' = m (Section 1.1 correctness, Section 3.1 proof);
  * Python's own integers (pow, divmod) and sympy's primality test, which
    are independent implementations;
  * invariants: 0, 1, N-1 are fixed by odd exponents; multiplicativity;
    CRT result equals the full-exponent result.
"""
import math
import os
import random

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split("=")
            vals[k] = int(v)
    return vals


def test_textbook_example():
    g = _golden("textbook_rsa_3233.txt")
    assert g["p"] * g["q"] == g["N"]
    assert (g["e"] * g["d"]) % g["phi"] == 1
    assert oracle.modexp(g["m"], g["e"], g["N"]) == g["c"]
    assert oracle.modexp(g["c"], g["d"], g["N"]) == g["m"]
    assert oracle.modinv(g["e"], g["phi"]) == g["d"]
    # CRT pieces of the same key
    p, q, d = g["p"], g["q"], g["d"]
    dp, dq, qinv = d % (p - 1), d % (q - 1), oracle.modinv(q, p)
    assert (qinv * q) % p == 1
    assert oracle.crt(g["c"], dp, dq, p, q, qinv) == g["m"]


def _odd_primes_below(n):
    return [x for x in range(3, n) if all(x % f for f in range(2, int(x ** 0.5) + 1))]


def test_bruteforce_tiny_moduli():
    """Every m in [0, N) for every pair of odd primes below 64."""
    primes = _odd_primes_below(64)
    checked = 0
    for i, p in enumerate(primes):
        for q in primes[i + 1:]:
            N, phi = p * q, (p - 1) * (q - 1)
            es = [e for e in (3, 5, 7, 17, 257) if math.gcd(e, phi) == 1][:2]
            m = np.arange(N, dtype=np.uint32).reshape(N, 1)
            for e in es:
                d = pow(e, -1, phi)
                c = oracle.modexp_chunks(m, np.array([[e]], np.uint32), np.array([[N]], np.uint32))
                # plain definition: e-fold repeated multiplication mod N
                ref = np.ones(N, np.int64)
                mm = np.arange(N, dtype=np.int64)
                for _ in range(e):
                    ref = (ref * mm) % N
                assert np.array_equal(c[:, 0].astype(np.int64), ref), (p, q, e)
                back = oracle.modexp_chunks(c, np.array([[d]], np.uint32), np.array([[N]], np.uint32))
                assert np.array_equal(back, m), (p, q, e)  # holds for all m: N is squarefree
                checked += N
    assert checked > 100000


@pytest.mark.parametrize("bits", [32, 64, 96, 512, 1024, 2048, 4096])
def test_modexp_vs_python_pow(bits):
    r = random.Random(bits)
    for _ in range(6 if bits >= 2048 else 25):
        N = r.getrandbits(bits) | (1 << (bits - 1))
        if r.random() < 0.5:
            N |= 1
        N = max(N, 2)
        x = r.getrandbits(bits + r.choice([0, 17, 64]))
        e = r.choice([1, 2, 3, 65537, r.getrandbits(r.choice([8, 64, bits]))]) or 1
        assert oracle.modexp(x, e, N) == pow(x, e, N), (bits, e)


def test_modexp_special_cases():
    N = (1 << 127) - 1  # a Mersenne prime
    for e in (1, 3, 65537, N - 2):
        assert oracle.modexp(0, e, N) == 0
        assert oracle.modexp(1, e, N) == 1
        if e % 2:
            assert oracle.modexp(N - 1, e, N) == N - 1
    assert oracle.modexp(N + 5, 1, N) == 5          # x is reduced first
    assert oracle.modexp(3, N - 1, N) == 1           # Fermat, N prime
    with pytest.raises(ValueError):
        oracle.modexp(3, 0, N)                       # e = 0 has no top bit
    # multiplicativity of x -> x^e mod N
    r = random.Random(5)
    for _ in range(20):
        a, b = r.getrandbits(120), r.getrandbits(120)
        e = r.getrandbits(100) | 1
        assert oracle.modexp(a * b, e, N) == oracle.mulmod(oracle.modexp(a, e, N), oracle.modexp(b, e, N), N)


def test_divmod_and_mulmod_vs_python():
    r = random.Random(11)
    patterns = [0, 1, 0xFFFFFFFF, 0x80000000, 0x7FFFFFFF]
    for _ in range(400):
        nu, nv = r.randint(1, 20), r.randint(1, 12)
        # structured limbs reach the rare correction branches of Algorithm D
        u = sum((r.choice(patterns) if r.random() < 0.6 else r.getrandbits(32)) << (32 * i) for i in range(nu))
        v = sum((r.choice(patterns) if r.random() < 0.6 else r.getrandbits(32)) << (32 * i) for i in range(nv)) or 7
        assert oracle.divmod_(u, v) == divmod(u, v)
        a, b = r.getrandbits(32 * nv), r.getrandbits(32 * nv)
        if v > 1:
            assert oracle.mulmod(a % v, b % v, v) == (a % v) * (b % v) % v
    # known add-back (step D6) cases in base 2^32
    for u, v in [((0x7FFFFFFF << 96) | (0x80000000 << 64), (0x80000000 << 64) | 1),
                 ((0x80000000 << 96) | (0xFFFFFFFE << 64), (0x80000000 << 64) | 0xFFFFFFFF << 32 | 0xFFFFFFFF)]:
        assert oracle.divmod_(u, v) == divmod(u, v)
    with pytest.raises(ZeroDivisionError):
        oracle.divmod_(5, 0)


def test_modinv_vs_python():
    r = random.Random(3)
    for bits in (16, 64, 256, 1024):
        for _ in range(10):
            m = r.getrandbits(bits) | 3
            a = r.getrandbits(bits) % m
            if math.gcd(a, m) == 1:
                assert oracle.modinv(a, m) == pow(a, -1, m)
            else:
                with pytest.raises(ValueError):
                    oracle.modinv(a, m)


@pytest.mark.parametrize("nbits,K", [(128, 4), (256, 3), (1024, 2)])
def test_keygen_properties(nbits, K):
    sympy = pytest.importorskip("sympy")
    keys = oracle.keygen(K, nbits, 65537, seed=1234 + nbits)
    seen = set()
    for k in range(K):
        kd = keys.key(k)
        p, q, N, d = kd["p"], kd["q"], kd["N"], kd["d"]
        for f in (p, q):
            assert sympy.isprime(f)
            assert f.bit_length() == nbits // 2 and (f >> (nbits // 2 - 2)) == 3
            assert math.gcd(65537, f - 1) == 1
        assert p != q and N == p * q and N.bit_length() == nbits
        phi = (p - 1) * (q - 1)
        assert d == pow(65537, -1, phi)
        assert kd["dp"] == d % (p - 1) and kd["dq"] == d % (q - 1)
        assert kd["qinv"] == pow(q, -1, p)
        seen.add(N)
    assert len(seen) == K
    again = oracle.keygen(K, nbits, 65537, seed=1234 + nbits)
    assert all(np.array_equal(again.a[n], keys.a[n]) for n in keys.a)
    other = oracle.keygen(1, nbits, 65537, seed=99)
    assert other.key(0)["N"] != keys.key(0)["N"]


def test_keygen_other_exponent():
    keys = oracle.keygen(2, 256, 3, seed=42)
    for k in range(2):
        kd = keys.key(k)
        phi = (kd["p"] - 1) * (kd["q"] - 1)
        assert (3 * kd["d"]) % phi == 1
    with pytest.raises(ValueError):
        oracle.keygen(1, 256, 4, seed=1)     # even exponent rejected
    with pytest.raises(ValueError):
        oracle.keygen(1, 200, 65537, seed=1)  # width not a multiple of 128


def test_crt_matches_full_exponent():
    keys = oracle.keygen(2, 512, 65537, seed=77)
    r = random.Random(8)
    for k in range(2):
        kd = keys.key(k)
        cs = [r.randrange(kd["N"]) for _ in range(12)] + [0, 1, kd["N"] - 1, kd["p"] * 5, kd["q"] * 7]
        for c in cs:
            full = pow(c, kd["d"], kd["N"])
            assert oracle.crt(c, kd["dp"], kd["dq"], kd["p"], kd["q"], kd["qinv"]) == full


# ---------------------------------------------------------------- multi-prime RSA (Section 2.1)

def _mp_key_from_primes(primes, e):
    """Key material of the multi-prime reading, computed with Python ints."""
    N = math.prod(primes)
    d = pow(e, -1, math.prod(r - 1 for r in primes))
    dexp = [d % (r - 1) for r in primes]
    coef = [pow(primes[1], -1, primes[0]), 0] + [pow(math.prod(primes[:i]), -1, primes[i]) for i in range(2, len(primes))]
    return N, d, dexp, coef


@pytest.mark.parametrize("primes,e", [((5, 7, 11), 7), ((11, 5, 7), 7), ((13, 3, 7, 11), 7), ((7, 11, 3, 5), 7),
                                      ((61, 53), 17)])
def test_crt_mp_bruteforce_tiny(primes, e):
    """Every message of tiny 2-, 3- and 4-prime moduli: the CRT recombination
    gives c^d mod N (Python pow) and inverts encryption (the RSA round trip)."""
    N, d, dexp, coef = _mp_key_from_primes(list(primes), e)
    for m in range(N):
        c = pow(m, e, N)
        assert oracle.crt_mp(c, list(primes), dexp, coef) == m
        assert oracle.crt_mp(m, list(primes), dexp, coef) == pow(m, d, N)


@pytest.mark.parametrize("nbits,b,K", [(384, 3, 3), (512, 4, 2), (768, 3, 2), (1024, 4, 1)])
def test_keygen_mp_properties(nbits, b, K):
    sympy = pytest.importorskip("sympy")
    keys = oracle.keygen_mp(K, nbits, b, 65537, seed=4321 + nbits + b)
    for k in range(K):
        r = keys.prime_list(k)
        N, d = oracle.from_limbs(keys.a["N"][k]), oracle.from_limbs(keys.a["d"][k])
        assert len(set(r)) == b
        for f in r:
            assert sympy.isprime(f) and f.bit_length() == nbits // b and math.gcd(65537, f - 1) == 1
        assert N == math.prod(r) and N.bit_length() == nbits
        N2, d2, dexp, coef = _mp_key_from_primes(r, 65537)
        assert d == d2
        assert keys.prime_list(k, "dexp") == dexp
        assert keys.prime_list(k, "coef") == coef
    again = oracle.keygen_mp(K, nbits, b, 65537, seed=4321 + nbits + b)
    assert all(np.array_equal(again.a[n], keys.a[n]) for n in keys.a)


def test_keygen_mp_two_primes_is_the_two_prime_key():
    two = oracle.keygen(3, 512, 65537, seed=31)
    mp = oracle.keygen_mp(3, 512, 2, 65537, seed=31)
    for k in range(3):
        kd = two.key(k)
        assert mp.prime_list(k) == [kd["p"], kd["q"]]
        assert mp.prime_list(k, "dexp") == [kd["dp"], kd["dq"]]
        assert mp.prime_list(k, "coef")[0] == kd["qinv"]
        assert oracle.from_limbs(mp.a["N"][k]) == kd["N"] and oracle.from_limbs(mp.a["d"][k]) == kd["d"]


def test_keygen_mp_argument_errors():
    for args in [(1, 768, 5), (1, 768, 1), (1, 512, 3), (1, 640, 4), (0, 768, 3)]:
        with pytest.raises(ValueError):
            oracle.keygen_mp(*args)


@pytest.mark.parametrize("nbits,b", [(768, 3), (1024, 4), (1536, 3)])
def test_crt_mp_matches_full_exponent(nbits, b):
    keys = oracle.keygen_mp(1, nbits, b, 65537, seed=17 + b)
    r = keys.prime_list(0)
    N, d = oracle.from_limbs(keys.a["N"][0]), oracle.from_limbs(keys.a["d"][0])
    rnd = random.Random(b)
    cs = [rnd.randrange(N) for _ in range(8)] + [0, 1, N - 1] + [f * 3 for f in r] + [N // r[0]]
    for c in cs:
        assert oracle.crt_mp(c, r, keys.prime_list(0, "dexp"), keys.prime_list(0, "coef")) == pow(c, d, N)
    s = nbits // 32
    m = np.stack([oracle.to_limbs(rnd.randrange(N), s) for _ in range(5)])
    assert np.array_equal(oracle.decrypt_chunks(m, keys, use_crt=True), oracle.decrypt_chunks(m, keys))


def test_chunk_loops_bind_key_t_mod_K():
    keys = oracle.keygen(3, 256, 65537, seed=5)
    r = random.Random(2)
    n = 11
    Ns = keys.ints("N")
    m = np.stack([oracle.to_limbs(r.randrange(Ns[t % 3]), 8) for t in range(n)])
    c = oracle.encrypt_chunks(m, keys)
    for t in range(n):
        assert oracle.from_limbs(c[t]) == pow(oracle.from_limbs(m[t]), 65537, Ns[t % 3])
    for use_crt in (False, True):
        back = oracle.decrypt_chunks(c, keys, use_crt=use_crt, threads=2)
        assert np.array_equal(back, m)


def test_split_join_definition():
    msg = bytes(range(1, 31)) + b"\xaa"          # 31 bytes, 128-bit keys -> P = 15
    ch = oracle.split(msg, 128)
    assert ch.shape == (3, 4)
    assert oracle.from_limbs(ch[0]) == int.from_bytes(bytes(range(1, 16)), "little")
    assert oracle.from_limbs(ch[1]) == int.from_bytes(bytes(range(16, 31)), "little")
    assert oracle.from_limbs(ch[2]) == 0xAA
    assert ch[0, 3] >> 24 == 0                     # the top byte of every chunk is zero
    assert oracle.join(ch, 31, 128) == msg
    assert oracle.split(b"", 1024).shape == (0, 32)
    assert oracle.join(np.zeros((0, 32), np.uint32), 0, 1024) == b""


@pytest.mark.parametrize("L,nbits,expected", [(32768, 1024, 259), (1048576, 2048, 4113), (104857600, 2048, 411207),
                                              (254, 2048, 1), (255, 2048, 1), (256, 2048, 2), (0, 2048, 0)])
def test_chunk_counts(L, nbits, expected):
    assert oracle.num_chunks(L, nbits) == expected


def test_split_join_roundtrip_random():
    r = np.random.default_rng(0)
    for nbits in (128, 1024, 2048):
        P = nbits // 8 - 1
        for L in [0, 1, P - 1, P, P + 1, 3 * P + 7, 1000]:
            msg = r.integers(0, 256, L, dtype=np.uint8).tobytes()
            ch = oracle.split(msg, nbits)
            assert ch.shape == (oracle.num_chunks(L, nbits), nbits // 32)
            assert all(oracle.from_limbs(row) < 1 << (8 * P) for row in ch)
            assert oracle.join(ch, L, nbits) == msg


def test_pmkrsa_roundtrip_message():
    """Section 3.1 correctness: join(decrypt(encrypt(split(M)))) = M with K key pairs."""
    keys = oracle.keygen(3, 512, 65537, seed=31)
    msg = np.random.default_rng(4).integers(0, 256, 1000, dtype=np.uint8).tobytes()
    ch = oracle.split(msg, 512)
    c = oracle.encrypt_chunks(ch, keys, threads=2)
    assert not np.array_equal(c, ch)
    Ns = keys.ints("N")
    assert all(oracle.from_limbs(c[t]) < Ns[t % 3] for t in range(len(c)))
    for use_crt in (False, True):
        assert oracle.join(oracle.decrypt_chunks(c, keys, use_crt=use_crt), len(msg), 512) == msg


def test_blinded_pmkrsa_algorithm1():
    """Algorithm 1 with the random matrix R: pinned against Python integers
    (c* = (m r)^e, c_r = r^e mod N) and the round trip of Section 3.1."""
    from paper_2111_11924_gb300.workloads import blinding_values

    keys = oracle.keygen(3, 512, 65537, seed=61)
    msg = np.random.default_rng(5).integers(0, 256, 700, dtype=np.uint8).tobytes()
    m = oracle.split(msg, 512)
    r = blinding_values(len(m), 512, seed=9)
    cstar, cr = oracle.blind_encrypt_chunks(m, r, keys, threads=2)
    Ns = keys.ints("N")
    for t in range(len(m)):
        N, mv, rv = Ns[t % 3], oracle.from_limbs(m[t]), oracle.from_limbs(r[t])
        assert oracle.from_limbs(cr[t]) == pow(rv, 65537, N)
        assert oracle.from_limbs(cstar[t]) == pow(mv * rv, 65537, N)
    back = oracle.blind_decrypt_chunks(cstar, cr, keys, threads=2)
    assert np.array_equal(back, m)
    assert oracle.join(back, len(msg), 512) == msg
    # the same ciphertext chunk blinded twice gives different c* (Section 3.4's point)
    r2 = blinding_values(len(m), 512, seed=10)
    cstar2, _ = oracle.blind_encrypt_chunks(m, r2, keys)
    assert not np.array_equal(cstar, cstar2)


def test_blinded_decrypt_rejects_non_invertible_r():
    keys = oracle.keygen(1, 256, 65537, seed=3)
    kd = keys.key(0)
    m = np.stack([oracle.to_limbs(5, 8)])
    cr = np.stack([oracle.to_limbs(kd["p"] * 3 % kd["N"], 8)])  # shares the factor p with N
    with pytest.raises(ValueError):
        oracle.blind_decrypt_chunks(m, cr, keys)


def test_keyed_chunk_loops_follow_an_explicit_key_map():
    """Explicit chunk-to-key map (the i x j reshape of Section 3.1 in any
    order): chunk t under key key_idx[t], checked with Python pow per chunk;
    the map t mod K gives the round-robin result."""
    K, nbits = 3, 256
    keys = oracle.keygen(K, nbits, 65537, 0x50444D4B0000C0DE)
    rng = np.random.default_rng(77)
    n = 40
    m = oracle.split(rng.integers(0, 256, n * (nbits // 8 - 1), dtype=np.uint8), nbits)
    idx = rng.integers(0, K, n)
    idx[:5] = 2  # a run on one key
    c = oracle.encrypt_chunks(m, keys, key_idx=idx)
    Ns, ds = keys.ints("N"), keys.ints("d")
    for t in range(n):
        assert oracle.from_limbs(c[t]) == pow(oracle.from_limbs(m[t]), 65537, Ns[idx[t]])
    back = oracle.decrypt_chunks(c, keys, key_idx=idx)
    assert np.array_equal(back, m)
    assert np.array_equal(oracle.decrypt_chunks(c, keys, use_crt=True, key_idx=idx), m)
    for t in (0, 17, n - 1):
        assert oracle.from_limbs(back[t]) == pow(oracle.from_limbs(c[t]), ds[idx[t]], Ns[idx[t]])
    assert np.array_equal(oracle.encrypt_chunks(m, keys, key_idx=np.arange(n) % K), oracle.encrypt_chunks(m, keys))
