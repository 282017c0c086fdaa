"""Multi-prime RSA (Section 2.1) through the C ABI against the oracle.

A multi-prime key has b distinct primes of n/b bits.  Encryption and full-d
decryption use N and d as before; CRT decryption runs one exponentiation
per prime over n/b bits and recombines the b residues.  Every result is
compared bit for bit: with the oracle's multi-prime CRT and its Algorithm 2
full-d decryption, with Python's pow, and with the library's own full-d
path.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2111_11924_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    import paper_2111_11924_gb300 as P

    return P


@pytest.fixture(scope="module")
def ctx(P):
    c = P.Context(0)
    yield c
    c.close()


def dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def host(t) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint32)


_keys = {}


def mp_keys(ctx, K, nbits, b, seed):
    """(library key set, oracle keys), the library's checked equal to the oracle's."""
    k = (K, nbits, b, seed)
    if k not in _keys:
        ks = ctx.keygen(K, nbits, 65537, seed, nprimes=b)
        ok = oracle.keygen_mp(K, nbits, b, 65537, seed)
        ex = ks.export()
        assert ks.nprimes == b
        for f in ok.a:
            assert np.array_equal(ex[f], ok.a[f]), f"multi-prime keygen mismatch in {f}"
        _keys[k] = (ks, ok)
    return _keys[k]


def checked_wide_mp_keys(ctx, K, nbits, b, seed):
    """Library keygen at widths where the oracle's keygen is slow; every key is
    verified with Python integers (Fermat probable primes, N = prod r_i of
    exactly nbits bits, e d = 1 mod phi, the CRT values)."""
    ks = ctx.keygen(K, nbits, 65537, seed, nprimes=b)
    ex = ks.export()
    h = nbits // 32 // b
    keys = []
    for k in range(K):
        r = [oracle.from_limbs(ex["primes"][k][i * h:(i + 1) * h]) for i in range(b)]
        dexp = [oracle.from_limbs(ex["dexp"][k][i * h:(i + 1) * h]) for i in range(b)]
        coef = [oracle.from_limbs(ex["coef"][k][i * h:(i + 1) * h]) for i in range(b)]
        N, d = oracle.from_limbs(ex["N"][k]), oracle.from_limbs(ex["d"][k])
        assert len(set(r)) == b and N == math.prod(r) and N.bit_length() == nbits
        for f in r:
            assert f.bit_length() == nbits // b and all(pow(x, f - 1, f) == 1 for x in (2, 3, 5, 7))
        assert (d * 65537) % math.prod(f - 1 for f in r) == 1
        assert dexp == [d % (f - 1) for f in r]
        assert (coef[0] * r[1]) % r[0] == 1 and coef[1] == 0
        assert all((coef[i] * math.prod(r[:i])) % r[i] == 1 for i in range(2, b))
        keys.append({"N": N, "d": d, "r": r})
    return ks, keys


def _edge_values(N, primes):
    vals = [0, 1, 2, N - 1, N - 2]
    for i, f in enumerate(primes):
        vals += [f, f * (3 + i), N // f]  # residues that vanish mod one prime / mod all but one
    return vals


@pytest.mark.parametrize("nbits,b,K,n", [(512, 4, 3, 61), (1024, 4, 4, 100), (2048, 4, 3, 45), (3072, 3, 2, 40),
                                         (4096, 4, 2, 16)])
def test_multiprime_crt_parity(ctx, nbits, b, K, n):
    ks, ok = mp_keys(ctx, K, nbits, b, seed=0x50444D4B0000E000 + nbits * 8 + b)
    s = nbits // 32
    rng = np.random.default_rng(nbits + b)
    Ns = ok.ints("N")
    m = np.stack([oracle.to_limbs(W.random_below(rng, Ns[t % K]), s) for t in range(n)])
    c = ctx.encrypt_chunks(ks, dev(m))
    assert np.array_equal(host(c), oracle.encrypt_chunks(m, ok, threads=8))
    crt = host(ctx.decrypt_chunks(ks, c, use_crt=True))
    assert np.array_equal(crt, m)
    assert np.array_equal(host(ctx.decrypt_chunks(ks, c)), m)
    # arbitrary values below N (not ciphertexts of chunks), including degenerate residues
    vals = []
    for t in range(n):
        k = t % K
        edge = _edge_values(Ns[k], ok.prime_list(k))
        vals.append(edge[t // K] if t // K < len(edge) else W.random_below(rng, Ns[k]))
    x = np.stack([oracle.to_limbs(v, s) for v in vals])
    got = host(ctx.decrypt_chunks(ks, dev(x), use_crt=True))
    assert np.array_equal(got, oracle.decrypt_chunks(x, ok, use_crt=True, threads=8))
    assert np.array_equal(got, host(ctx.decrypt_chunks(ks, dev(x))))
    for t in range(0, n, 7):
        kd = ok.key(t % K)
        assert oracle.from_limbs(got[t]) == pow(vals[t], kd["d"], kd["N"]), t
    assert ctx.status() == 0


@pytest.mark.parametrize("nbits,b", [(3072, 3), (4096, 4), (2048, 4)])
def test_multiprime_every_geometry(ctx, P, nbits, b):
    ks, ok = mp_keys(ctx, 2, nbits, b, seed=0x50444D4B0000E100 + nbits + b)
    s, h = nbits // 32, nbits // 32 // b
    rng = np.random.default_rng(5 + b)
    m = np.stack([oracle.to_limbs(W.random_below(rng, N), s) for N in ok.ints("N") * 9])
    c = ctx.encrypt_chunks(ks, dev(m))
    ref = oracle.decrypt_chunks(host(c)[:4], ok, use_crt=True)
    assert np.array_equal(ref, m[:4])
    configs = P.kernel_configs(h, True)
    assert configs
    for window in (5, 4):  # the full and the small odd-power table
        for tpi, form in configs:
            ctx.set_kernel_config(h, True, tpi, form)
            ctx.set_kernel_window(h, True, window)
            try:
                got = host(ctx.decrypt_chunks(ks, c, use_crt=True))
            finally:
                ctx.set_kernel_config(h, True, 0)
                ctx.set_kernel_window(h, True, 0)
            assert np.array_equal(got, m), (tpi, form, window)


@pytest.mark.parametrize("nbits,b", [(6144, 3), (6144, 4), (8192, 4)])
def test_multiprime_wide_keys(ctx, nbits, b):
    ks, keys = checked_wide_mp_keys(ctx, 2, nbits, b, seed=0x50444D4B0000E200 + nbits + b)
    s = nbits // 32
    rng = np.random.default_rng(nbits + b)
    vals = [W.random_below(rng, keys[t % 2]["N"]) for t in range(6)]
    m = np.stack([oracle.to_limbs(v, s) for v in vals])
    c = ctx.encrypt_chunks(ks, dev(m))
    ch = host(c)
    for t in range(6):
        assert oracle.from_limbs(ch[t]) == oracle.modexp(vals[t], 65537, keys[t % 2]["N"]), t
    assert np.array_equal(host(ctx.decrypt_chunks(ks, c, use_crt=True)), m)
    k0 = keys[0]
    x = [k0["r"][0] * 5, k0["N"] - 1, W.random_below(rng, k0["N"])]
    xx = np.zeros((5, s), np.uint32)  # chunks 0, 2, 4 use key 0
    for j, v in enumerate(x):
        xx[2 * j] = oracle.to_limbs(v, s)
    got = host(ctx.decrypt_chunks(ks, dev(xx), use_crt=True))
    for j, v in enumerate(x):
        assert oracle.from_limbs(got[2 * j]) == pow(v, k0["d"], k0["N"]), j
    assert ctx.status() == 0


def test_multiprime_message_roundtrip_and_host_calls(ctx):
    nbits, b = 3072, 3
    ks, ok = mp_keys(ctx, 4, nbits, b, seed=0x50444D4B0000E300)
    msg = np.random.default_rng(3).integers(0, 256, 50_000, dtype=np.uint8)
    d_msg = torch.from_numpy(msg).cuda()
    ch = ctx.split(nbits, d_msg)
    c = ctx.encrypt_chunks(ks, ch)
    assert np.array_equal(host(c), oracle.encrypt_chunks(oracle.split(msg, nbits), ok, threads=8))
    plain = ctx.decrypt_chunks(ks, c, use_crt=True)
    assert bytes(ctx.join(nbits, plain, len(msg)).cpu().numpy()) == msg.tobytes()
    h_msg = torch.from_numpy(msg).pin_memory()
    h_c = torch.empty(tuple(c.shape), dtype=torch.int32).pin_memory()
    ctx.encrypt_message_host(ks, h_msg, h_c)
    assert torch.equal(h_c, c.cpu())
    back = torch.zeros(len(msg), dtype=torch.uint8).pin_memory()
    ctx.decrypt_message_host(ks, h_c, back, use_crt=True)
    assert torch.equal(back, h_msg)


@pytest.mark.parametrize("nbits,b", [(1024, 4), (3072, 3)])
def test_multiprime_blinded(ctx, P, nbits, b):
    """Algorithm 1 with R on multi-prime keys: C*, C_R equal the oracle's, and
    decryption (c* c_r^-1)^d with the inverse and the power both by CRT over
    the b primes recovers every chunk; an r sharing a prime is reported."""
    K = 3
    ks, ok = mp_keys(ctx, K, nbits, b, seed=0x50444D4B0000E400 + nbits)
    msg = np.random.default_rng(nbits).integers(0, 256, 9000, dtype=np.uint8)
    m = oracle.split(msg, nbits)
    r = W.blinding_values(len(m), nbits, seed=0x50444D4B0000E500 + nbits)
    cstar_ref, cr_ref = oracle.blind_encrypt_chunks(m, r, ok, threads=8)
    cstar, cr = ctx.encrypt_blinded(ks, dev(m), dev(r))
    assert np.array_equal(host(cstar), cstar_ref) and np.array_equal(host(cr), cr_ref)
    for use_crt in (False, True):
        assert np.array_equal(host(ctx.decrypt_blinded(ks, cstar, cr, use_crt=use_crt)), m), use_crt
    assert ctx.status() == 0
    bad = host(cr).copy()
    r2 = ok.prime_list(0)[b - 1]
    bad[K] = oracle.to_limbs(r2 * 7, nbits // 32)  # chunk K (key 0) shares the prime r_{b-1} with N_0
    out = host(ctx.decrypt_blinded(ks, cstar, dev(bad), use_crt=True))
    assert ctx.status() == P.pmkrsa.PMK_ENOINV
    assert np.array_equal(np.delete(out, K, axis=0), np.delete(m, K, axis=0))


@pytest.mark.parametrize("direct_max", [256, 0])
def test_multiprime_in_a_batch(ctx, P, direct_max):
    """A batch mixing multi-prime CRT jobs (3 and 4 primes) with two-prime
    jobs replays bit-identical to one call per job, as grid launches per job
    and through the persistent queues (one task per prime)."""
    from paper_2111_11924_gb300 import pmkrsa as B

    a, oka = mp_keys(ctx, 3, 3072, 3, seed=0x50444D4B0000E600)
    c4, okc = mp_keys(ctx, 2, 2048, 4, seed=0x50444D4B0000E700)
    two = ctx.keygen(2, 2048, 65537, 0x50444D4B0000E800)
    rng = np.random.default_rng(11)
    jobs = []
    for ks, Ns, n, op in [(a, oka.ints("N"), 29, B.OP_DECRYPT_CRT), (c4, okc.ints("N"), 17, B.OP_DECRYPT_CRT),
                          (two, None, 13, B.OP_DECRYPT_CRT), (a, oka.ints("N"), 5, B.OP_ENCRYPT),
                          (c4, okc.ints("N"), 9, B.OP_DECRYPT)]:
        s = ks.nbits // 32
        if Ns is None:
            x = np.zeros((n, s), np.uint32)
            x[:, : s - 1] = rng.integers(0, 2**32, (n, s - 1), dtype=np.uint64).astype(np.uint32)
        else:
            x = np.stack([oracle.to_limbs(W.random_below(rng, Ns[t % len(Ns)]), s) for t in range(n)])
        jobs.append((ks, dev(x), torch.zeros((n, s), dtype=torch.int32, device="cuda"), op))
    ctx.set_batch_direct_max(direct_max)
    try:
        batch = ctx.batch(jobs)
    finally:
        ctx.set_batch_direct_max(256)
    assert (batch.n_tasks > 0) == (direct_max == 0)
    batch.launch()
    ctx.check()
    for ks, x, out, op in jobs:
        ref = ctx.encrypt_chunks(ks, x) if op == B.OP_ENCRYPT else ctx.decrypt_chunks(ks, x, use_crt=op == B.OP_DECRYPT_CRT)
        assert torch.equal(out, ref), (ks.nbits, ks.nprimes, op)
    ks, x, out, op = jobs[0]
    assert np.array_equal(host(out)[:5], oracle.decrypt_chunks(host(x)[:5], oka))
    batch.destroy()
    two.free()


def test_multiprime_autotune_and_errors(ctx, P):
    ks, ok = mp_keys(ctx, 2, 2048, 4, seed=0x50444D4B0000E900)
    res = ctx.autotune(ks, 200, "crt", reps=1)
    assert (res["tpi"], res["form"]) in P.kernel_configs(16, True)
    ctx.set_kernel_config(16, True, 0)
    with pytest.raises(P.PMKError) as ei:  # valid multi-prime width, but no 24-limb full-width kernel is built
        ctx.keygen(1, 768, 65537, 1, nprimes=3)
    assert ei.value.code == P.pmkrsa.PMK_EUNSUPPORTED
    for args in [(1, 2048, 3), (1, 768, 5), (1, 768, 1), (1, 640, 4), (0, 768, 3), (16384, 768, 3)]:
        with pytest.raises(P.PMKError) as ei:
            ctx.keygen(args[0], args[1], 65537, 1, nprimes=args[2])
        assert ei.value.code == P.pmkrsa.PMK_EINVAL, args
    # the two-prime export fields do not describe a multi-prime key
    lib = P.load_library()
    buf = np.zeros(2 * 2048 // 32, np.uint32)
    p32 = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    assert lib.pmk_keyset_export_fields(ks.handle, None, None, p32, None, None, None, None) == P.pmkrsa.PMK_EINVAL


def test_multiprime_keyset_from_oracle_primes(ctx, P):
    """Importing the oracle's primes gives the oracle's key material, and the
    imported set decrypts like the generated one; malformed primes are rejected."""
    ok = oracle.keygen_mp(3, 3072, 3, 65537, 0x50444D4B0000EB00)
    ks = ctx.keyset_from_primes_multi(3072, 3, 65537, ok.a["primes"])
    ex = ks.export()
    for f in ok.a:
        assert np.array_equal(ex[f], ok.a[f]), f
    rng = np.random.default_rng(4)
    m = np.stack([oracle.to_limbs(W.random_below(rng, N), 96) for N in ok.ints("N") * 4])
    c = ctx.encrypt_chunks(ks, dev(m))
    assert np.array_equal(host(c), oracle.encrypt_chunks(m, ok))
    assert np.array_equal(host(ctx.decrypt_chunks(ks, c, use_crt=True)), m)
    bad = ok.a["primes"].copy()
    bad[0, 32:64] = bad[0, 0:32]  # r_1 = r_0
    with pytest.raises(P.PMKError):
        ctx.keyset_from_primes_multi(3072, 3, 65537, bad)
    bad = ok.a["primes"].copy()
    bad[1, 0] &= ~np.uint32(1)  # an even "prime"
    with pytest.raises(P.PMKError):
        ctx.keyset_from_primes_multi(3072, 3, 65537, bad)
    ks.free()


@pytest.mark.parametrize("nbits,b,K,n,e", [(1024, 4, 1, 9, 65537), (3072, 3, 5, 3, 65537), (2048, 4, 2, 11, 3),
                                           (512, 4, 3, 1, 17)])
def test_multiprime_degenerate_counts_and_exponents(ctx, nbits, b, K, n, e):
    """One key, fewer chunks than keys, small public exponents; encryption in
    place; CRT and full d against the oracle."""
    ks = ctx.keygen(K, nbits, e, 0x50444D4B0000ED00 + nbits + K, nprimes=b)
    ok = oracle.keygen_mp(K, nbits, b, e, 0x50444D4B0000ED00 + nbits + K)
    ex = ks.export()
    assert all(np.array_equal(ex[f], ok.a[f]) for f in ok.a)
    rng = np.random.default_rng(n)
    Ns = ok.ints("N")
    m = np.stack([oracle.to_limbs(W.random_below(rng, Ns[t % K]), nbits // 32) for t in range(n)])
    x = dev(m)
    ctx.encrypt_chunks(ks, x, out=x)  # in place
    assert np.array_equal(host(x), oracle.encrypt_chunks(m, ok))
    for use_crt in (True, False):
        assert np.array_equal(host(ctx.decrypt_chunks(ks, x, use_crt=use_crt)), m), use_crt
    assert ctx.status() == 0
    ks.free()


def test_maximum_key_count(ctx, P):
    """16,383 keys, the most a key set takes: with 4 primes the CRT grid has
    65,532 rows (the CUDA limit is 65,535).  Every key's chunks round-trip
    and a sample matches Python pow."""
    K = 16383
    for nbits, b in ((512, 4), (128, 2)):
        ks = ctx.keygen(K, nbits, 65537, 0x50444D4B0000F000 + nbits, nprimes=b)
        ex = ks.export()
        s = nbits // 32
        n = K + 17
        rng = np.random.default_rng(nbits)
        m = rng.integers(0, 2**32, (n, s), dtype=np.uint64).astype(np.uint32)
        m[:, -1] = 0  # below every modulus
        c = ctx.encrypt_chunks(ks, dev(m))
        for use_crt in (True, False):
            assert np.array_equal(host(ctx.decrypt_chunks(ks, c, use_crt=use_crt)), m), (nbits, use_crt)
        ch = host(c)
        for t in (0, 1, K - 1, K, n - 1):
            N = oracle.from_limbs(ex["N"][t % K])
            assert oracle.from_limbs(ch[t]) == pow(oracle.from_limbs(m[t]), 65537, N), (nbits, t)
        assert ctx.status() == 0
        ks.free()
