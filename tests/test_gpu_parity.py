"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Integer results are compared bit-exactly: a modular exponentiation has one
correct residue.  Key material on the oracle side comes from the oracle's own
keygen and is checked equal to the library's.
"""
import ctypes

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


def keys_for(ctx, K, nbits, seed, e=65537):
    """(library key set, oracle keys) for the same seeded key initialisation."""
    k = (K, nbits, seed, e)
    if k not in _keys:
        ks = ctx.keygen(K, nbits, e, seed)
        ok = oracle.keygen(K, nbits, e, seed)
        ex = ks.export()
        for f in ok.a:
            assert np.array_equal(ex[f], ok.a[f]), f"keygen mismatch in {f}"
        _keys[k] = (ks, ok)
    return _keys[k]


# ------------------------------------------------------------------ split / join

@pytest.mark.parametrize("nbits", [128, 1024, 2048, 4096])
def test_split_join_parity(ctx, nbits):
    P = nbits // 8 - 1
    rng = np.random.default_rng(nbits)
    for L in [1, 2, 3, P - 1, P, P + 1, 3 * P + 7, 4099, 32768]:
        msg = rng.integers(0, 256, L, dtype=np.uint8)
        d_msg = torch.from_numpy(msg).cuda()
        ch = ctx.split(nbits, d_msg)
        assert np.array_equal(host(ch), oracle.split(msg, nbits)), L
        back = ctx.join(nbits, dev(oracle.split(msg, nbits)), L)
        assert bytes(back.cpu().numpy()) == msg.tobytes()
        assert bytes(ctx.join(nbits, ch, L).cpu().numpy()) == msg.tobytes()


@pytest.mark.parametrize("off", [1, 3, 4, 8, 15])
def test_split_join_unaligned_message(ctx, off):
    """A message (or join output) that starts off a 16-byte boundary takes the
    byte-wise path and still gives the oracle's chunks."""
    nbits = 1024
    rng = np.random.default_rng(off)
    for L in [5, 127, 128, 1000]:
        msg = rng.integers(0, 256, L, dtype=np.uint8)
        base = torch.zeros(L + 16, dtype=torch.uint8, device="cuda")
        base[off:off + L] = torch.from_numpy(msg).cuda()
        ch = ctx.split(nbits, base[off:off + L])
        assert np.array_equal(host(ch), oracle.split(msg, nbits)), (off, L)
        out = torch.zeros(L + 16, dtype=torch.uint8, device="cuda")
        ctx.join(nbits, ch, L, out=out[off:off + L])
        o = out.cpu().numpy()
        assert bytes(o[off:off + L]) == msg.tobytes()
        assert not o[:off].any() and not o[off + L:].any()  # nothing written outside the message


def test_split_join_empty(ctx, P):
    d_msg = torch.empty(0, dtype=torch.uint8, device="cuda")
    ch = ctx.split(2048, d_msg)
    assert ch.shape == (0, 64)
    assert ctx.join(2048, ch, 0).numel() == 0


def test_split_join_full_1mib(ctx):
    w = W.FILE_1MIB_2048
    msg = w.message()
    ch = ctx.split(w.nbits, torch.from_numpy(msg).cuda())
    assert np.array_equal(host(ch), oracle.split(msg, w.nbits))
    assert bytes(ctx.join(w.nbits, ch, len(msg)).cpu().numpy()) == msg.tobytes()


# ------------------------------------------------------------------ small widths, edge values

@pytest.mark.parametrize("nbits,K", [(128, 3), (256, 2), (512, 2)])
def test_edge_values_small_widths(ctx, nbits, K):
    ks, ok = keys_for(ctx, K, nbits, seed=900 + nbits)
    s = nbits // 32
    Ns = ok.ints("N")
    rng = np.random.default_rng(nbits)
    vals = []
    for t in range(24 * K):
        N = Ns[t % K]
        pick = t // K
        special = [0, 1, 2, N - 1, N - 2, N // 2, (1 << (nbits - 1)) % N, ok.key(t % K)["p"], ok.key(t % K)["q"]]
        vals.append(special[pick] if pick < len(special) else W.random_below(rng, N))
    m = np.stack([oracle.to_limbs(v, s) for v in vals])
    c_ref = oracle.encrypt_chunks(m, ok)
    c = ctx.encrypt_chunks(ks, dev(m))
    assert np.array_equal(host(c), c_ref)
    for use_crt in (False, True):
        ref = oracle.decrypt_chunks(c_ref, ok, use_crt=use_crt)
        got = ctx.decrypt_chunks(ks, dev(c_ref), use_crt=use_crt)
        assert np.array_equal(host(got), ref), use_crt
        assert np.array_equal(ref, m)  # the oracle's own round trip
    assert ctx.status() == 0


# ------------------------------------------------------------------ the 32 KiB / 1024-bit workload, every chunk

def test_small_workload_every_chunk(ctx):
    w = W.SMALL_1024
    ks, ok = keys_for(ctx, w.K, w.nbits, w.key_seed)
    msg = w.message()
    m = oracle.split(msg, w.nbits)
    assert m.shape[0] == w.n_chunks == 259
    d_m = ctx.split(w.nbits, torch.from_numpy(msg).cuda())
    c = ctx.encrypt_chunks(ks, d_m)
    c_ref = oracle.encrypt_chunks(m, ok, threads=8)
    assert np.array_equal(host(c), c_ref)
    for use_crt in (False, True):
        d = ctx.decrypt_chunks(ks, c, use_crt=use_crt)
        assert np.array_equal(host(d), oracle.decrypt_chunks(c_ref, ok, use_crt=use_crt, threads=8)), use_crt
        assert bytes(ctx.join(w.nbits, d, len(msg)).cpu().numpy()) == msg.tobytes()
    assert ctx.status() == 0


# ------------------------------------------------------------------ the 1 MiB / 2048-bit workload (bench configuration)

def test_1mib_2048_encrypt_all_decrypt_sampled(ctx):
    w = W.FILE_1MIB_2048
    ks, ok = keys_for(ctx, w.K, w.nbits, w.key_seed)
    msg = w.message()
    m = oracle.split(msg, w.nbits)
    d_m = ctx.split(w.nbits, torch.from_numpy(msg).cuda())
    c = ctx.encrypt_chunks(ks, d_m)
    c_host = host(c)
    assert np.array_equal(c_host, oracle.encrypt_chunks(m, ok, threads=8))   # every chunk
    d_full = ctx.decrypt_chunks(ks, c, use_crt=False)
    d_crt = ctx.decrypt_chunks(ks, c, use_crt=True)
    full_h, crt_h = host(d_full), host(d_crt)
    assert np.array_equal(full_h, m)        # round trip on every chunk
    assert np.array_equal(crt_h, full_h)    # CRT identical to full-d on every chunk
    # sampled chunks through the oracle's own decryption (both forms), incl. the ragged last chunk
    rng = np.random.default_rng(7)
    idx = np.unique(np.concatenate([rng.choice(w.n_chunks, 56, replace=False), [0, 1, w.n_chunks - 1]]))
    sub = np.ascontiguousarray(c_host[idx])
    # keep each chunk bound to its own key: build a K-row key table per sampled chunk
    for use_crt, got in ((False, full_h), (True, crt_h)):
        for t in idx[:24] if use_crt else idx:
            k = int(t) % w.K
            kd = ok.key(k)
            cv = oracle.from_limbs(c_host[t])
            ref = oracle.crt(cv, kd["dp"], kd["dq"], kd["p"], kd["q"], kd["qinv"]) if use_crt else \
                oracle.modexp(cv, kd["d"], kd["N"])
            assert oracle.from_limbs(got[t]) == ref, (t, use_crt)
    assert sub.shape[0] == len(idx)
    assert ctx.status() == 0


# ------------------------------------------------------------------ launch geometries

@pytest.mark.parametrize("nbits,crt", [(2048, False), (2048, True), (1024, False), (1024, True), (4096, False),
                                       (3072, True), (3072, False)])
def test_every_kernel_geometry(ctx, P, nbits, crt):
    """Every compiled (lanes, form) geometry gives the same bit-exact result;
    for the CRT residues also with the small odd-power table (window <= 4).
    Each geometry runs in both of its instantiations: round robin, and over
    key groups (explicit key indices in a random order, checked against the
    oracle with the same indices)."""
    K = 3
    ks, ok = keys_for(ctx, K, nbits, seed=4242 + nbits)
    rng = np.random.default_rng(1)
    Ns = ok.ints("N")
    n = 37  # ragged: several blocks per key and a partial one
    vals = [W.random_below(rng, Ns[t % K]) for t in range(n)]
    # edge values among them: 0, 1, 2, N - 1, N - 2 and all-ones low limbs, for every product form
    for t, f in ((6, lambda N: 0), (7, lambda N: 1), (8, lambda N: 2), (9, lambda N: N - 1), (10, lambda N: N - 2),
                 (11, lambda N: (1 << (nbits - 2)) - 1)):
        vals[t] = f(Ns[t % K])
    c = np.stack([oracle.to_limbs(v, nbits // 32) for v in vals])
    ref = oracle.decrypt_chunks(c[:12], ok)
    idx = rng.integers(0, K, n)  # explicit key indices: chunk t under key idx[t]
    c2 = np.stack([oracle.to_limbs(W.random_below(rng, Ns[k]), nbits // 32) for k in idx])
    ref2 = oracle.decrypt_chunks(c2[:12], ok, key_idx=idx[:12])
    d_idx = torch.from_numpy(idx.astype(np.int32)).cuda()
    limbs = nbits // 64 if crt else nbits // 32
    configs = P.kernel_configs(limbs, crt)
    assert len(configs) >= 1
    outs, outs2, tried = [], [], []
    for window in ((5, 4) if crt else (5,)):
        for tpi, form in configs:
            ctx.set_kernel_config(limbs, crt, tpi, form)
            ctx.set_kernel_window(limbs, crt, window)
            try:
                outs.append(host(ctx.decrypt_chunks(ks, dev(c), use_crt=crt)))
                outs2.append(host(ctx.decrypt_chunks(ks, dev(c2), use_crt=crt, key_idx=d_idx)))
                tried.append((tpi, form, window))
            finally:
                ctx.set_kernel_config(limbs, crt, 0)
                ctx.set_kernel_window(limbs, crt, 0)
    for o, o2, cfg in zip(outs, outs2, tried):
        assert np.array_equal(o[:12], ref), cfg
        assert np.array_equal(o, outs[0]), cfg
        assert np.array_equal(o2[:12], ref2), cfg
        assert np.array_equal(o2, outs2[0]), cfg
    assert ctx.get_kernel_config(limbs, crt)[0] in {t for t, _ in configs}
    assert ctx.get_kernel_window(limbs, crt) == 5


def test_window_bound_api_batch_and_autotune(ctx, P):
    """The window bound is validated and read back; the per-call kernels, the
    persistent batch kernels and the autotuner honour it; no result changes."""
    from paper_2111_11924_gb300 import pmkrsa as B

    for bad in (1, 3, 6):
        with pytest.raises(B.PMKError) as ei:
            ctx.set_kernel_window(32, True, bad)
        assert ei.value.code == B.PMK_EINVAL
    for limbs, crt in ((40, True), (64, False)):  # no kernel / no small-table kernel
        with pytest.raises(B.PMKError) as ei:
            ctx.set_kernel_window(limbs, crt, 4)
        assert ei.value.code == B.PMK_EUNSUPPORTED
    assert ctx.get_kernel_window(64, False) == 5 and ctx.get_kernel_window(32, True) == 5
    ks, ok = keys_for(ctx, 3, 2048, seed=4242 + 2048)
    rng = np.random.default_rng(5)
    Ns = ok.ints("N")
    n = 70
    c = dev(np.stack([oracle.to_limbs(W.random_below(rng, Ns[t % 3]), 64) for t in range(n)]))
    full5, crt5 = ctx.decrypt_chunks(ks, c), ctx.decrypt_chunks(ks, c, use_crt=True)
    assert torch.equal(full5, crt5)
    assert np.array_equal(host(full5)[:4], oracle.decrypt_chunks(host(c)[:4], ok))
    try:
        ctx.set_kernel_window(32, True, 4)
        assert ctx.get_kernel_window(32, True) == 4
        assert torch.equal(ctx.decrypt_chunks(ks, c, use_crt=True), full5)
        for tpi, form in P.kernel_configs(32, True):  # every geometry; those without a small build use the full table
            ctx.set_kernel_config(32, True, tpi, form)
            assert torch.equal(ctx.decrypt_chunks(ks, c, use_crt=True), full5), (tpi, form)
        ctx.set_kernel_config(32, True, 0)
        for direct_max in (256, 0):  # grid launches per job, then the persistent queues
            outs = [torch.zeros_like(c) for _ in range(3)]
            ctx.set_batch_direct_max(direct_max)
            batch = ctx.batch([(ks, c, outs[0], B.OP_DECRYPT), (ks, c, outs[1], B.OP_DECRYPT_CRT),
                               (ks, full5, outs[2], B.OP_ENCRYPT)])
            assert (batch.n_tasks > 0) == (direct_max == 0)
            batch.launch()
            ctx.check()
            assert torch.equal(outs[0], full5) and torch.equal(outs[1], full5) and torch.equal(outs[2], c)
            batch.destroy()
        ctx.set_batch_direct_max(256)
        for mode in ("decrypt", "crt"):
            res = ctx.autotune(ks, n, mode, reps=1)
            limbs = 32 if mode == "crt" else 64
            assert res["window"] in ((4, 5) if mode == "crt" else (5,))
            assert ctx.get_kernel_window(limbs, mode == "crt") == res["window"]
            assert torch.equal(ctx.decrypt_chunks(ks, c, use_crt=(mode == "crt")), full5)
    finally:
        for limbs, crt in ((64, False), (32, True)):
            ctx.set_kernel_window(limbs, crt, 0)
            ctx.set_kernel_config(limbs, crt, 0)


@pytest.mark.parametrize("nbits", [3072, 4096])
def test_wide_keys(ctx, nbits):
    ks, ok = keys_for(ctx, 2, nbits, seed=77 + nbits)
    rng = np.random.default_rng(nbits)
    Ns = ok.ints("N")
    m = np.stack([oracle.to_limbs(W.random_below(rng, Ns[t % 2]), nbits // 32) for t in range(6)])
    c = ctx.encrypt_chunks(ks, dev(m))
    c_ref = oracle.encrypt_chunks(m, ok)
    assert np.array_equal(host(c), c_ref)
    assert np.array_equal(host(ctx.decrypt_chunks(ks, c)), m)
    assert np.array_equal(host(ctx.decrypt_chunks(ks, c, use_crt=True)), m)
    d0 = ok.key(0)
    assert oracle.from_limbs(host(ctx.decrypt_chunks(ks, c))[0]) == oracle.modexp(oracle.from_limbs(c_ref[0]), d0["d"], d0["N"])


# ------------------------------------------------------------------ degenerate cases and errors

def test_degenerate_counts_and_inplace(ctx):
    ks, ok = keys_for(ctx, 5, 512, seed=31)
    Ns = ok.ints("N")
    rng = np.random.default_rng(3)
    for n in (1, 3, 5, 6):  # fewer chunks than keys, exactly K, K + 1
        m = np.stack([oracle.to_limbs(W.random_below(rng, Ns[t % 5]), 16) for t in range(n)])
        d_m = dev(m)
        ctx.encrypt_chunks(ks, d_m, out=d_m)  # in place
        assert np.array_equal(host(d_m), oracle.encrypt_chunks(m, ok))
        ctx.decrypt_chunks(ks, d_m, out=d_m)  # in place, full d
        assert np.array_equal(host(d_m), m)
    empty = torch.empty((0, 16), dtype=torch.int32, device="cuda")
    ctx.encrypt_chunks(ks, empty)
    ctx.decrypt_chunks(ks, empty, use_crt=True)
    assert ctx.status() == 0


def test_out_of_range_chunk_reported(ctx, P):
    ks, ok = keys_for(ctx, 2, 256, seed=8)
    Ns = ok.ints("N")
    vals = [5, Ns[1], 7, (1 << 256) - 1, Ns[0] - 1, Ns[1] + 1]
    m = np.stack([oracle.to_limbs(v, 8) for v in vals])
    out = ctx.decrypt_chunks(ks, dev(m))
    assert ctx.status() == P.pmkrsa.PMK_ERANGE
    assert ctx.status() == 0  # cleared
    got = host(out)
    for t in (0, 2, 4):
        kd = ok.key(t % 2)
        assert oracle.from_limbs(got[t]) == oracle.modexp(vals[t], kd["d"], kd["N"])
    ctx.encrypt_chunks(ks, dev(m[:2]))
    assert ctx.status() == P.pmkrsa.PMK_ERANGE


def test_failing_chunk_is_attributed(ctx, P):
    """pmk_sync_status_detail names the smallest failing chunk of the call:
    a range error (chunk >= its modulus), a key index >= K, and a blinding
    value sharing a prime with its modulus; and none after clearing."""
    ks, ok = keys_for(ctx, 3, 512, seed=31)
    rng = np.random.default_rng(31)
    m = oracle.split(rng.integers(0, 256, 400 * 63, dtype=np.uint8), 512)
    bad = m.copy()
    for t in (271, 90, 305):  # three bad chunks; 90 is the first
        bad[t] = ok.a["N"][t % 3]
    ctx.encrypt_chunks(ks, dev(bad))
    assert ctx.status_detail() == (P.pmkrsa.PMK_ERANGE, 90)
    assert ctx.status_detail() == (P.pmkrsa.PMK_OK, None)
    idx = rng.integers(0, 3, m.shape[0]).astype(np.uint32)
    idx[[333, 17]] = 9
    ctx.encrypt_chunks(ks, dev(m), key_idx=dev(idx))
    assert ctx.status_detail() == (P.pmkrsa.PMK_EKEYINDEX, 17)
    # blinded decryption: r of chunk 44 is a multiple of key (44 mod 3)'s first prime
    c = ctx.encrypt_chunks(ks, dev(m))
    r = oracle.split(rng.integers(0, 256, 400 * 63, dtype=np.uint8), 512)
    r[44] = oracle.to_limbs(3 * oracle.from_limbs(ok.a["p"][44 % 3]), 16)
    cstar, cr = ctx.encrypt_blinded(ks, c, dev(r))
    ctx.decrypt_blinded(ks, cstar, cr, use_crt=True)
    assert ctx.status_detail() == (P.pmkrsa.PMK_ENOINV, 44)


def test_argument_errors(ctx, P):
    ks, _ = keys_for(ctx, 2, 256, seed=8)
    m = torch.zeros((4, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(P.PMKError):
        ctx.decrypt_chunks(ks, m, use_crt=True, out=m)  # CRT in place is rejected
    with pytest.raises(P.PMKError):
        ctx.keygen(1, 200)  # width not a multiple of 128
    with pytest.raises(P.PMKError):
        ctx.keygen(1, 256, e=4)
    lib = P.load_library()
    import ctypes
    assert lib.pmk_split(ctx.handle, 2048, ctypes.c_void_p(m.data_ptr()), 1000, ctypes.c_void_p(m.data_ptr()), 3,
                         None) == P.pmkrsa.PMK_EINVAL  # 1000 bytes need 4 chunks


def test_host_buffer_calls_and_from_primes(ctx):
    w = W.SMALL_1024
    ks, ok = keys_for(ctx, w.K, w.nbits, w.key_seed)
    msg = torch.from_numpy(w.message()).pin_memory()
    cipher = torch.empty((w.n_chunks, w.limbs), dtype=torch.int32).pin_memory()
    ctx.encrypt_message_host(ks, msg, cipher)
    ref = oracle.encrypt_chunks(oracle.split(msg.numpy(), w.nbits), ok, threads=8)
    assert np.array_equal(cipher.numpy().view(np.uint32), ref)
    back = torch.empty(w.msg_bytes, dtype=torch.uint8).pin_memory()
    for use_crt in (False, True):
        back.zero_()
        ctx.decrypt_message_host(ks, cipher, back, use_crt=use_crt)
        assert torch.equal(back, msg)
    ks2 = ctx.keyset_from_primes(w.nbits, w.e, ok.a["p"], ok.a["q"])
    ex = ks2.export()
    assert all(np.array_equal(ex[f], ok.a[f]) for f in ok.a)


@pytest.mark.parametrize("mode", ["encrypt", "decrypt", "crt"])
def test_autotune_chooses_a_built_geometry(ctx, P, mode):
    ks, ok = keys_for(ctx, 2, 1024, seed=555)
    res = ctx.autotune(ks, 300, mode, reps=1)
    limbs = 16 if mode == "crt" else 32
    assert (res["tpi"], res["form"]) in P.kernel_configs(limbs, mode == "crt")
    assert res["ms"] > 0
    assert ctx.get_kernel_config(limbs, mode == "crt") == (res["tpi"], res["form"])
    rng = np.random.default_rng(9)
    m = np.stack([oracle.to_limbs(W.random_below(rng, N), 32) for N in ok.ints("N") * 5])
    c = ctx.encrypt_chunks(ks, dev(m))
    assert np.array_equal(host(c), oracle.encrypt_chunks(m, ok))
    assert np.array_equal(host(ctx.decrypt_chunks(ks, c, use_crt=(mode == "crt"))), m)
    ctx.set_kernel_config(limbs, mode == "crt", 0)


def _checked_wide_keys(ctx, K, nbits, seed):
    """Library keygen at widths where the oracle's keygen takes minutes; every
    key is verified here with Python integers instead (N = pq, e d = 1 mod phi,
    Fermat probable primes, CRT values)."""
    ks = ctx.keygen(K, nbits, 65537, seed)
    ex = ks.export()
    keys = []
    for k in range(K):
        v = {f: oracle.from_limbs(ex[f][k]) for f in ex}
        p, q, N, d = v["p"], v["q"], v["N"], v["d"]
        assert N == p * q and N.bit_length() == nbits and p != q
        phi = (p - 1) * (q - 1)
        assert (d * 65537) % phi == 1
        for f in (p, q):
            assert f.bit_length() == nbits // 2 and all(pow(b, f - 1, f) == 1 for b in (2, 3, 5, 7))
        assert v["dp"] == d % (p - 1) and v["dq"] == d % (q - 1) and (v["qinv"] * q) % p == 1
        keys.append(v)
    return ks, keys


@pytest.mark.parametrize("nbits", [6144, 8192])
def test_6144_8192_bit_keys(ctx, P, nbits):
    ks, keys = _checked_wide_keys(ctx, 2, nbits, seed=0x50444D4B00008000 + nbits)
    s = nbits // 32
    rng = np.random.default_rng(nbits)
    vals = [W.random_below(rng, keys[t % 2]["N"]) for t in range(5)]
    m = np.stack([oracle.to_limbs(v, s) for v in vals])
    c = host(ctx.encrypt_chunks(ks, dev(m)))
    for t in range(5):
        assert oracle.from_limbs(c[t]) == oracle.modexp(vals[t], 65537, keys[t % 2]["N"]), t
    k0 = keys[0]
    ref0 = oracle.modexp(oracle.from_limbs(c[0]), k0["d"], k0["N"])
    assert ref0 == vals[0]
    for crt in (False, True):
        limbs = s // 2 if crt else s
        for tpi, form in P.kernel_configs(limbs, crt):
            ctx.set_kernel_config(limbs, crt, tpi, form)
            try:
                got = host(ctx.decrypt_chunks(ks, dev(c), use_crt=crt))
            finally:
                ctx.set_kernel_config(limbs, crt, 0)
            assert np.array_equal(got, m), (crt, tpi, form)
            assert oracle.from_limbs(got[0]) == ref0
    assert ctx.status() == 0


@pytest.mark.parametrize("queued", [False, True])
def test_batched_persistent_graph_matches_per_call(ctx, P, queued):
    """A mixed batch (five key sets at 512-4096 bits, encrypt / full d / CRT,
    ragged sizes) replayed from its CUDA graph equals one call per job, bit
    for bit, and keeps doing so when the input contents change between
    launches.  Every job of both launches is also checked against the oracle
    on a sample of at least 8 chunks that includes its last one.  Queued:
    the context's direct-launch limit is 0, so the small jobs go through the
    persistent queues; otherwise every job is its own grid launch."""
    from paper_2111_11924_gb300 import pmkrsa as B

    sets = [keys_for(ctx, K, nb, seed=700 + nb) for K, nb in ((3, 1024), (2, 2048), (5, 512))]
    wide = []  # library keys at 3072 / 4096 bits, checked with Python integers; the oracle computes with them
    for K, nb, seed in ((2, 4096, 0x50444D4B0000B000), (3, 3072, 0x50444D4B0000B100)):
        ks_w, keys_w = _checked_wide_keys(ctx, K, nb, seed=seed)
        wide.append((ks_w, keys_w, oracle.OracleKeys(K, nb, 65537, ks_w.export())))
    rng = np.random.default_rng(77)

    def chunks_for(Ns, n, s):
        return np.stack([oracle.to_limbs(W.random_below(rng, Ns[t % len(Ns)]), s) for t in range(n)])

    def key_set(si):
        if si < 3:
            ks, ok = sets[si]
            return ks, ok, ok.ints("N")
        ks_w, keys_w, ok_w = wide[si - 3]
        return ks_w, ok_w, [k["N"] for k in keys_w]

    jobs = []
    plan = [(0, 41, B.OP_DECRYPT), (0, 7, B.OP_ENCRYPT), (1, 33, B.OP_DECRYPT_CRT), (2, 3, B.OP_DECRYPT),
            (1, 1, B.OP_DECRYPT), (2, 90, B.OP_ENCRYPT), (3, 5, B.OP_DECRYPT_CRT), (3, 4, B.OP_DECRYPT),
            (4, 12, B.OP_DECRYPT), (4, 9, B.OP_DECRYPT_CRT), (4, 10, B.OP_ENCRYPT)]
    for si, n, op in plan:
        ks, _, Ns = key_set(si)
        x = dev(chunks_for(Ns, n, ks.nbits // 32))
        jobs.append((ks, x, torch.zeros_like(x), op))
    ctx.set_batch_direct_max(0 if queued else 256)
    try:
        batch = ctx.batch(jobs)
    finally:
        ctx.set_batch_direct_max(256)
    if queued:
        assert batch.n_kernels >= 4 and batch.n_tasks > 0
    else:
        assert batch.n_tasks == 0 and batch.n_kernels == len(jobs)
    for rep in range(2):
        if rep == 1:  # new contents, same buffers
            for (ks, x, out, op), (si, n, _) in zip(jobs, plan):
                x.copy_(dev(chunks_for(key_set(si)[2], n, ks.nbits // 32)))
        for _, _, out, _ in jobs:
            out.zero_()
        batch.launch()
        ctx.check()
        for (ks, x, out, op), (si, n, _) in zip(jobs, plan):
            if op == B.OP_ENCRYPT:
                ref = ctx.encrypt_chunks(ks, x)
            else:
                ref = ctx.decrypt_chunks(ks, x, use_crt=(op == B.OP_DECRYPT_CRT))
            assert torch.equal(out, ref), (ks.nbits, op, n)
            ok = key_set(si)[1]
            sample = np.unique(np.concatenate([rng.choice(n, min(n, 8), replace=False), [n - 1]]))
            xin = host(x)[sample]
            want = (oracle.encrypt_chunks(xin, ok, key_idx=sample % ok.K) if op == B.OP_ENCRYPT
                    else oracle.decrypt_chunks(xin, ok, key_idx=sample % ok.K))
            assert np.array_equal(host(out)[sample], want), (ks.nbits, op, n, rep)
    batch.destroy()


@pytest.mark.parametrize("nbits,K,length", [(512, 3, 3000), (2048, 8, 61200), (2048, 8, 400000)])
def test_blinded_algorithm1_parity(ctx, nbits, K, length):
    """Algorithm 1 with the random matrix R: GPU C*, C_R equal the oracle's bit
    for bit; GPU decryption (c* c_r^-1)^d (full d and CRT) recovers every chunk,
    and so does the oracle's literal r' = c_r^d, m* = c*^d, m* r'^-1."""
    ks, ok = keys_for(ctx, K, nbits, seed=0x50444D4B0000D000 + nbits)
    msg = np.random.default_rng(nbits).integers(0, 256, length, dtype=np.uint8)
    m = oracle.split(msg, nbits)
    r = W.blinding_values(len(m), nbits, seed=0x50444D4B0000D100 + nbits)
    cstar_ref, cr_ref = oracle.blind_encrypt_chunks(m, r, ok, threads=8)
    cstar, cr = ctx.encrypt_blinded(ks, dev(m), dev(r))
    assert np.array_equal(host(cstar), cstar_ref)
    assert np.array_equal(host(cr), cr_ref)
    for use_crt in (False, True):
        back = ctx.decrypt_blinded(ks, cstar, cr, use_crt=use_crt)
        assert np.array_equal(host(back), m), use_crt
    sample = slice(0, 10)
    assert np.array_equal(oracle.blind_decrypt_chunks(cstar_ref[sample], cr_ref[sample], ok, threads=8), m[sample])
    assert ctx.status() == 0


@pytest.mark.parametrize("nbits,K", [(512, 3), (2048, 4)])
def test_blinded_values_across_their_whole_range(ctx, nbits, K):
    """Algorithm 1 allows any r in Z*_N.  Blinding values at the top of the
    range -- N - 1, N - 2, and random values in [2^(n-8), N) -- and at the
    bottom (1, 2): C*, C_R equal the oracle's, and both decryption paths
    (full d, and CRT: the fused joint exponentiation at 2048 bits, Fermat
    inverses and recombination at 512 bits) recover every chunk."""
    ks, ok = keys_for(ctx, K, nbits, seed=0x50444D4B0000D200 + nbits)
    Ns = ok.ints("N")
    s = nbits // 32
    rng = np.random.default_rng(nbits + 5)
    n = 40
    m = oracle.split(rng.integers(0, 256, n * (nbits // 8 - 1), dtype=np.uint8), nbits)
    vals = []
    for t in range(n):
        N = Ns[t % K]
        special = {0: N - 1, 1: N - 2, 2: 1, 3: 2, 4: N - 1, 5: N - 2}
        if t in special:
            vals.append(special[t])
        else:  # uniform in [2^(n-8), N): above what the default blinding generator draws
            lo = 1 << (nbits - 8)
            vals.append(lo + W.random_below(rng, N - lo))
    r = np.stack([oracle.to_limbs(v, s) for v in vals])
    assert all(v >= 1 << (nbits - 8) for t, v in enumerate(vals) if t not in (2, 3))
    cstar_ref, cr_ref = oracle.blind_encrypt_chunks(m, r, ok, threads=8)
    cstar, cr = ctx.encrypt_blinded(ks, dev(m), dev(r))
    assert np.array_equal(host(cstar), cstar_ref)
    assert np.array_equal(host(cr), cr_ref)
    for use_crt in (False, True):
        back = ctx.decrypt_blinded(ks, cstar, cr, use_crt=use_crt)
        assert np.array_equal(host(back), m), use_crt
    assert np.array_equal(oracle.blind_decrypt_chunks(cstar_ref[:8], cr_ref[:8], ok, threads=8), m[:8])
    assert ctx.status() == 0


def test_blinded_non_invertible_value_reported(ctx, P):
    ks, ok = keys_for(ctx, 2, 256, seed=8)
    k0 = ok.key(0)
    m = np.stack([oracle.to_limbs(v, 8) for v in (5, 6, 7, 8)])
    r = np.stack([oracle.to_limbs(v, 8) for v in (3, 4, 5, 6)])
    cstar, cr = ctx.encrypt_blinded(ks, dev(m), dev(r))
    assert ctx.status() == 0
    bad = host(cr).copy()
    bad[2] = oracle.to_limbs(k0["p"] * 11, 8)  # chunk 2 (key 0) shares the factor p with N_0
    for use_crt in (False, True):  # the inverse-then-power path and the fused joint exponentiation
        out = ctx.decrypt_blinded(ks, cstar, dev(bad), use_crt=use_crt)
        assert ctx.status() == P.pmkrsa.PMK_ENOINV, use_crt
        got = host(out)
        for t in (0, 1, 3):
            assert oracle.from_limbs(got[t]) == oracle.from_limbs(m[t]), (use_crt, t)


@pytest.mark.parametrize("nbits", [1024, 2048])
def test_thread_per_chunk_baseline_matches(ctx, nbits):
    ks, ok = keys_for(ctx, 3, nbits, seed=321 + nbits)
    rng = np.random.default_rng(nbits + 1)
    Ns = ok.ints("N")
    m = np.stack([oracle.to_limbs(W.random_below(rng, Ns[t % 3]), nbits // 32) for t in range(40)])
    c_base = ctx.modexp_chunks_baseline(ks, dev(m), decrypt=False)
    c = ctx.encrypt_chunks(ks, dev(m))
    assert torch.equal(c_base, c)
    assert np.array_equal(host(c)[:8], oracle.encrypt_chunks(m[:8], ok))
    d_base = ctx.modexp_chunks_baseline(ks, c, decrypt=True)
    assert np.array_equal(host(d_base), m)
    assert ctx.status() == 0


@pytest.mark.parametrize("e", [3, 17, 257])
def test_other_public_exponents(ctx, e):
    """Small public exponents change the encryption schedule (e = 3 and 17 use
    the odd-power table) and d; results must still match the oracle."""
    ks, ok = keys_for(ctx, 3, 1024, seed=2000 + e, e=e)
    rng = np.random.default_rng(e)
    Ns = ok.ints("N")
    m = np.stack([oracle.to_limbs(W.random_below(rng, Ns[t % 3]), 32) for t in range(20)])
    c = ctx.encrypt_chunks(ks, dev(m))
    assert np.array_equal(host(c), oracle.encrypt_chunks(m, ok))
    for use_crt in (False, True):
        assert np.array_equal(host(ctx.decrypt_chunks(ks, c, use_crt=use_crt)), m)
    assert np.array_equal(host(ctx.decrypt_chunks(ks, c))[:5], oracle.decrypt_chunks(host(c)[:5], ok))
    ctx.set_kernel_window(16, True, 4)  # CRT schedules within 4-bit windows
    try:
        assert np.array_equal(host(ctx.decrypt_chunks(ks, c, use_crt=True)), m)
    finally:
        ctx.set_kernel_window(16, True, 0)


def test_100mib_roundtrip_and_oracle_sample(ctx):
    """The 100 MiB / K=16 / 2048-bit file: the whole-file round trip on the
    GPU (full d and CRT), and a seeded 4,096-chunk sample of the ciphertext
    checked chunk by chunk against the oracle."""
    w = W.FILE_100MIB_2048
    ks, ok = keys_for(ctx, w.K, w.nbits, w.key_seed)
    msg = w.message()
    d_msg = torch.from_numpy(msg).cuda()
    m = ctx.split(w.nbits, d_msg)
    assert m.shape[0] == w.n_chunks == 411207
    c = ctx.encrypt_chunks(ks, m)
    back = ctx.join(w.nbits, ctx.decrypt_chunks(ks, c, use_crt=True), w.msg_bytes)
    assert torch.equal(back, d_msg)
    back_full = ctx.decrypt_chunks(ks, c)
    assert torch.equal(back_full, m)
    idx = np.sort(np.random.default_rng(0x50444D4B).choice(w.n_chunks, 4096, replace=False))
    m_h, c_h = host(m)[idx], host(c)[idx]
    # chunk t uses key t mod K: group the sample by key
    for k in range(w.K):
        sel = idx % w.K == k
        sub_keys = oracle.OracleKeys(1, w.nbits, w.e, {f: ok.a[f][k:k + 1] for f in ok.a})
        assert np.array_equal(oracle.encrypt_chunks(m_h[sel], sub_keys, threads=8), c_h[sel]), k
    assert np.array_equal(m_h, oracle.split(msg, w.nbits)[idx])
    assert ctx.status() == 0


def test_integer_peak_measurements_are_sane(ctx):
    """The roofline denominators come from the library's own loops: the MAC
    rate and the mad.lo rate per clock per SM must be positive, below the
    architectural issue limit of 128 lanes per clock per SM, and consistent
    with each other (a MAC costs at least one mad.lo-equivalent issue)."""
    mac = ctx.measure_int_peak()
    lo = ctx.measure_imad_peak()
    assert mac["num_sms"] == lo["num_sms"] > 0
    assert 1.0 < mac["macs_per_clk_per_sm"] <= 128.0
    assert 1.0 < lo["mad_lo_per_clk_per_sm"] <= 128.0
    assert mac["macs_per_clk_per_sm"] <= lo["mad_lo_per_clk_per_sm"] * 1.05
    assert mac["sm_mhz"] > 100 and lo["sm_mhz"] > 100


def test_batch_large_jobs_take_a_grid_launch(ctx, P):
    """With the direct-launch limit below the batch's job count (here 0),
    jobs that fill the GPU at least once still run as plain grid launches
    inside the batch graph, next to queued small jobs; every output equals
    the per-call result, and a batch of one large job holds no queued
    tasks."""
    from paper_2111_11924_gb300 import pmkrsa as B

    ks = ctx.keygen(8, 2048, 65537, 0x50444D4B0000EC00)
    msg = torch.from_numpy(np.random.default_rng(12).integers(0, 256, 30000 * 255, dtype=np.uint8)).cuda()
    big = ctx.encrypt_chunks(ks, ctx.split(2048, msg))            # 30,000 chunks
    small = big[:37].clone()
    jobs = [(ks, big[:20000], torch.zeros_like(big[:20000]), B.OP_DECRYPT_CRT),
            (ks, big, torch.zeros_like(big), B.OP_DECRYPT),
            (ks, small, torch.zeros_like(small), B.OP_DECRYPT_CRT)]
    ctx.set_batch_direct_max(0)
    try:
        batch = ctx.batch(jobs)
        one_out = torch.zeros_like(big)
        one = ctx.batch([(ks, big, one_out, B.OP_DECRYPT_CRT)])
    finally:
        ctx.set_batch_direct_max(256)
    assert batch.n_kernels >= 3 and batch.n_tasks > 0
    batch.launch()
    ctx.check()
    for k, x, out, op in jobs:
        assert torch.equal(out, ctx.decrypt_chunks(k, x, use_crt=op == B.OP_DECRYPT_CRT)), (x.shape[0], op)
    assert torch.equal(jobs[1][2], ctx.split(2048, msg))
    batch.destroy()
    assert one.n_tasks == 0 and one.n_kernels == 1
    one.launch()
    ctx.check()
    assert torch.equal(one_out, ctx.split(2048, msg))
    one.destroy()
    ks.free()


def _guarded(n_words, fill=0x5A5A5A5A):
    """A device int32 buffer of n_words with 1024-word guard zones on both
    sides filled with `fill`; returns (whole buffer, interior slice)."""
    g = 1024
    buf = torch.full((n_words + 2 * g,), fill - (1 << 32) if fill >= (1 << 31) else fill, dtype=torch.int32,
                     device="cuda")
    return buf, buf[g:g + n_words]


def _guards_intact(buf, n_words, fill=0x5A5A5A5A):
    g = 1024
    torch.cuda.synchronize()
    h = buf.cpu().numpy().view(np.uint32)
    return bool((h[:g] == fill).all() and (h[g + n_words:] == fill).all())


def test_canary_words_around_every_output(ctx, P):
    """Every kernel writes only inside its output: guard zones around the
    device buffers (a stand-in for a sanitizer, which this pool does not run)
    keep their pattern through split, encrypt, full-d and CRT decrypt (2 and
    3 primes), blinded encrypt / decrypt, the batch graph and join."""
    from paper_2111_11924_gb300 import pmkrsa as B

    for nbits, b in ((2048, 2), (3072, 3)):
        ks = ctx.keygen(3, nbits, 65537, 0x50444D4B0000EE00 + nbits, nprimes=b)
        s = nbits // 32
        L = 12345
        msg = np.random.default_rng(nbits).integers(0, 256, L, dtype=np.uint8)
        n = oracle.num_chunks(L, nbits)
        mbuf = torch.full((L + 8192,), 0x5A, dtype=torch.uint8, device="cuda")
        d_msg = mbuf[4096:4096 + L]
        d_msg.copy_(torch.from_numpy(msg).cuda())
        cb, chunks = _guarded(n * s)
        ctx.split(nbits, d_msg, out=chunks.view(n, s))
        xb, cipher = _guarded(n * s)
        ctx.encrypt_chunks(ks, chunks.view(n, s), out=cipher.view(n, s))
        for use_crt in (False, True):
            pb, plain = _guarded(n * s)
            ctx.decrypt_chunks(ks, cipher.view(n, s), use_crt=use_crt, out=plain.view(n, s))
            assert _guards_intact(pb, n * s), (nbits, use_crt)
            assert torch.equal(plain, chunks)
        r = torch.from_numpy(W.blinding_values(n, nbits, 9).view(np.int32)).cuda()
        sb, cstar = _guarded(n * s)
        rb, cr = _guarded(n * s)
        ctx.encrypt_blinded(ks, chunks.view(n, s), r, out_cstar=cstar.view(n, s), out_cr=cr.view(n, s))
        assert _guards_intact(sb, n * s) and _guards_intact(rb, n * s)
        bb, bl = _guarded(n * s)
        ctx.decrypt_blinded(ks, cstar.view(n, s), cr.view(n, s), use_crt=True, out=bl.view(n, s))
        assert _guards_intact(bb, n * s) and torch.equal(bl, chunks)
        for direct_max in (256, 0):  # the batch as a grid launch, then through the persistent queue
            qb, qout = _guarded(n * s)
            ctx.set_batch_direct_max(direct_max)
            batch = ctx.batch([(ks, cipher.view(n, s), qout.view(n, s), B.OP_DECRYPT_CRT)])
            ctx.set_batch_direct_max(256)
            assert (batch.n_tasks > 0) == (direct_max == 0)
            batch.launch()
            ctx.check()
            assert _guards_intact(qb, n * s) and torch.equal(qout, chunks), direct_max
            batch.destroy()
        obuf = torch.full((L + 8192,), 0x5A, dtype=torch.uint8, device="cuda")
        ctx.join(nbits, chunks.view(n, s), L, out=obuf[4096:4096 + L])
        o = obuf.cpu().numpy()
        assert (o[:4096] == 0x5A).all() and (o[4096 + L:] == 0x5A).all()
        assert bytes(o[4096:4096 + L]) == msg.tobytes()
        for buf in (cb, xb):
            assert _guards_intact(buf, n * s)
        assert ctx.status() == 0
        ks.free()


def test_chunk_count_bound(ctx, P):
    ks, _ = keys_for(ctx, 2, 512, seed=3)
    x = torch.zeros((4, 16), dtype=torch.int32, device="cuda")
    rc = P.load_library().pmk_encrypt_chunks(ctx.handle, ks.handle, ctypes.c_void_p(x.data_ptr()),
                                             ctypes.c_void_p(x.data_ptr()), 1 << 32, None, None)
    assert rc == P.pmkrsa.PMK_EINVAL


def test_autotune_cache_applies_stored_geometry(ctx, P, tmp_path):
    ks, ok = keys_for(ctx, 2, 1024, seed=556)
    cache = P.TuneCache(str(tmp_path / "tune.json"))
    first = ctx.autotune(ks, 300, "decrypt", reps=1, cache=cache)
    assert "cached" not in first
    ctx.set_kernel_config(32, False, 0)
    second = ctx.autotune(ks, 300, "decrypt", reps=1, cache=P.TuneCache(str(tmp_path / "tune.json")))
    assert second["cached"] and (second["tpi"], second["form"]) == (first["tpi"], first["form"])
    assert ctx.get_kernel_config(32, False) == (first["tpi"], first["form"])
    ctx.set_kernel_config(32, False, 0)


def test_sharded_message_through_the_library(ctx):
    """The shards of one message, each split / encrypted / decrypted / joined
    on its own (as one rank per GPU would, here one after another on one
    GPU), give the whole message's ciphertext chunks and plaintext."""
    from paper_2111_11924_gb300 import sharding as SH

    w = W.FILE_1MIB_2048
    ks, ok = keys_for(ctx, w.K, w.nbits, w.key_seed)
    msg = torch.from_numpy(w.message()).cuda()
    whole = ctx.encrypt_chunks(ks, ctx.split(w.nbits, msg))
    parts, back = [], []
    for sh in SH.shards(w.msg_bytes, w.nbits, w.K, 5):
        piece = msg[sh.byte_lo:sh.byte_hi]
        c = ctx.encrypt_chunks(ks, ctx.split(w.nbits, piece))
        parts.append(c)
        back.append(ctx.join(w.nbits, ctx.decrypt_chunks(ks, c, use_crt=True), sh.n_bytes))
    assert torch.equal(torch.cat(parts), whole)
    assert torch.equal(torch.cat(back), msg)
