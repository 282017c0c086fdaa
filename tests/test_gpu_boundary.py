"""The boundary's key handling on the GPU: explicit chunk-to-key indices (the
d_key_idx argument of pmk_encrypt_chunks and pmk_decrypt_chunks) against the
oracle, and key sets restored from their serialised blob.

Section 3.1 reshapes the chunks into an i x j matrix with one row per key;
the order of the fill is the caller's.  With d_key_idx the library groups
chunks by key on the device and every result must equal the oracle's
c_t = m_t^e mod N_k, m_t = c_t^d mod N_k with k = key_idx[t], chunk by chunk.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    import oracle
    import paper_2111_11924_gb300 as P

    ctx = P.Context(0)
    yield P, oracle, ctx
    ctx.close()


def _setup(P, oracle, ctx, K, nbits, n, seed, nprimes=2):
    ks = ctx.keygen(K, nbits, 65537, seed, nprimes=nprimes)
    ok = oracle.keygen(K, nbits, 65537, seed) if nprimes == 2 else oracle.keygen_mp(K, nbits, nprimes, 65537, seed)
    rng = np.random.default_rng(seed & 0xFFFF)
    msg = rng.integers(0, 256, n * (nbits // 8 - 1) - 7, dtype=np.uint8)  # ragged last chunk
    m = oracle.split(msg, nbits)
    return ks, ok, m, rng


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


@pytest.mark.parametrize("nbits,K,n,pattern", [
    (1024, 5, 1000, "skewed"),      # most chunks on key 0, key 3 empty
    (1024, 5, 1000, "rows"),        # the i x j matrix filled row by row: a contiguous run per key
    (512, 7, 333, "random"),
    (2048, 8, 700, "random"),
    (3072, 4, 129, "single"),       # every chunk on one key
])
def test_key_index_every_chunk_matches_oracle(env, nbits, K, n, pattern):
    P, oracle, ctx = env
    ks, ok, m, rng = _setup(P, oracle, ctx, K, nbits, n, 0x50444D4B0000E000 + nbits + K + n)
    n = m.shape[0]
    if pattern == "skewed":
        idx = np.where(rng.random(n) < 0.7, 0, rng.choice([1, 2, 4], n))
    elif pattern == "rows":
        idx = np.minimum(np.arange(n) // -(-n // K), K - 1)
    elif pattern == "single":
        idx = np.full(n, K - 1)
    else:
        idx = rng.integers(0, K, n)
    idx = idx.astype(np.uint32)
    d_idx = _dev(idx)
    c_ref = oracle.encrypt_chunks(m, ok, threads=8, key_idx=idx)
    c = ctx.encrypt_chunks(ks, _dev(m), key_idx=d_idx)
    ctx.check()
    assert np.array_equal(c.cpu().numpy().view(np.uint32), c_ref)
    for use_crt in (False, True):
        back = ctx.decrypt_chunks(ks, c, use_crt=use_crt, key_idx=d_idx)
        ctx.check()
        assert np.array_equal(back.cpu().numpy().view(np.uint32), m), use_crt
    # the oracle's own decryption of a sample, including the last chunk
    sample = np.unique(np.concatenate([rng.choice(n, 24, replace=False), [n - 1]]))
    d_ref = oracle.decrypt_chunks(c_ref[sample], ok, key_idx=idx[sample])
    assert np.array_equal(d_ref, m[sample])
    ks.free()


def test_key_index_where_the_kernels_differ_in_block_size(env):
    """4096-bit keys: the CRT residue kernel holds 16 instances per block and
    the recombination 8, so the key-group table is aligned to the larger;
    random and one-key maps give the oracle's results for full d and CRT
    (the oracle computes with the library's exported keys)."""
    P, oracle, ctx = env
    K, nbits = 4, 4096
    ks = ctx.keygen(K, nbits, 65537, 0x50444D4B0000E800)
    ok = oracle.OracleKeys(K, nbits, 65537, ks.export())
    rng = np.random.default_rng(48)
    n = 301
    m = oracle.split(rng.integers(0, 256, n * (nbits // 8 - 1) - 11, dtype=np.uint8), nbits)
    for idx in (rng.integers(0, K, n), np.full(n, 2)):
        idx = idx.astype(np.uint32)
        d_idx = _dev(idx)
        c = ctx.encrypt_chunks(ks, _dev(m), key_idx=d_idx)
        ctx.check()
        assert np.array_equal(c.cpu().numpy().view(np.uint32), oracle.encrypt_chunks(m, ok, threads=8, key_idx=idx))
        for use_crt in (False, True):
            back = ctx.decrypt_chunks(ks, c, use_crt=use_crt, key_idx=d_idx)
            ctx.check()
            assert np.array_equal(back.cpu().numpy().view(np.uint32), m), use_crt
    ks.free()


def test_key_index_round_robin_map_equals_null(env):
    """key_idx[t] = t mod K reproduces the call without indices bit for bit,
    in place as well."""
    P, oracle, ctx = env
    ks, ok, m, _ = _setup(P, oracle, ctx, 6, 1024, 900, 0x50444D4B0000E100)
    n = m.shape[0]
    d_m = _dev(m)
    d_idx = _dev((np.arange(n) % 6).astype(np.uint32))
    plain = ctx.encrypt_chunks(ks, d_m)
    keyed = ctx.encrypt_chunks(ks, d_m, key_idx=d_idx)
    assert torch.equal(plain, keyed)
    buf = keyed.clone()
    ctx.decrypt_chunks(ks, buf, out=buf, key_idx=d_idx)  # in place, full d
    ctx.check()
    assert torch.equal(buf, d_m)
    ks.free()


def test_key_index_out_of_range_is_reported(env):
    """An index >= K is reported as PMK_EKEYINDEX; its chunk's output is left
    as it was and every other chunk is still exact."""
    P, oracle, ctx = env
    ks, ok, m, rng = _setup(P, oracle, ctx, 3, 512, 200, 0x50444D4B0000E200)
    n = m.shape[0]
    idx = rng.integers(0, 3, n).astype(np.uint32)
    idx[[7, 150]] = [3, 0xFFFFFFFF]
    out = torch.full((n, 16), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    ctx.encrypt_chunks(ks, _dev(m), out=out, key_idx=_dev(idx))
    assert ctx.status() == P.pmkrsa.PMK_EKEYINDEX
    assert ctx.status() == P.pmkrsa.PMK_OK  # reported once, then cleared
    got = out.cpu().numpy().view(np.uint32)
    good = np.setdiff1d(np.arange(n), [7, 150])
    assert np.array_equal(got[good], oracle.encrypt_chunks(m[good], ok, key_idx=idx[good]))
    assert (got[[7, 150]] == 0x5A5A5A5A).all()
    ks.free()


def test_key_index_multiprime_crt(env):
    """Explicit indices with a 3-prime key set: CRT over three residues per
    chunk, each under its own key."""
    P, oracle, ctx = env
    ks, ok, m, rng = _setup(P, oracle, ctx, 4, 3072, 200, 0x50444D4B0000E300, nprimes=3)
    idx = rng.integers(0, 4, m.shape[0]).astype(np.uint32)
    d_idx = _dev(idx)
    c = ctx.encrypt_chunks(ks, _dev(m), key_idx=d_idx)
    assert np.array_equal(c.cpu().numpy().view(np.uint32), oracle.encrypt_chunks(m, ok, threads=8, key_idx=idx))
    back = ctx.decrypt_chunks(ks, c, use_crt=True, key_idx=d_idx)
    ctx.check()
    assert np.array_equal(back.cpu().numpy().view(np.uint32), m)
    ks.free()


def test_key_index_many_keys_and_empty_segments(env):
    """300 keys, most without chunks: the segment offsets and the block-to-key
    search stay exact when many segments are empty."""
    P, oracle, ctx = env
    ks, ok, m, rng = _setup(P, oracle, ctx, 300, 256, 500, 0x50444D4B0000E400)
    idx = rng.choice([0, 1, 150, 298, 299], m.shape[0]).astype(np.uint32)
    c = ctx.encrypt_chunks(ks, _dev(m), key_idx=_dev(idx))
    ctx.check()
    assert np.array_equal(c.cpu().numpy().view(np.uint32), oracle.encrypt_chunks(m, ok, key_idx=idx))
    ks.free()


def test_blob_import_on_device_decrypts_alike(env):
    """A key set exported as a blob and imported on the device holds the same
    key material and gives the same ciphertexts and plaintexts."""
    P, oracle, ctx = env
    for K, nbits, b in ((4, 2048, 2), (2, 3072, 3)):
        ks = ctx.keygen(K, nbits, 65537, 0x50444D4B0000E500 + b, nprimes=b)
        blob = ks.export_blob()
        ks2 = ctx.import_keyset(blob)
        ex, ex2 = ks.export(), ks2.export()
        assert all(np.array_equal(ex[f], ex2[f]) for f in ex)
        assert ks2.export_blob() == blob
        m = oracle.split(np.random.default_rng(b).integers(0, 256, 40_000, dtype=np.uint8), nbits)
        d_m = _dev(m)
        c1, c2 = ctx.encrypt_chunks(ks, d_m), ctx.encrypt_chunks(ks2, d_m)
        assert torch.equal(c1, c2)
        assert torch.equal(ctx.decrypt_chunks(ks2, c1, use_crt=True), d_m)
        ctx.check()
        ks.free()
        ks2.free()


def test_buffers_of_another_shape_and_host_only_keys_are_refused(env):
    """The binding refuses, before any launch, chunk buffers whose width is
    not the key set's or whose length differs from the input's, a message
    buffer of another length, and a key-index vector of another length; the
    library refuses a host-only key set (EINVAL) in the device calls."""
    P, oracle, ctx = env
    ks = ctx.keygen(2, 2048, 65537, 0x50444D4B0000E700)
    good = torch.zeros((5, 64), dtype=torch.int32, device="cuda")
    narrow = torch.zeros((5, 32), dtype=torch.int32, device="cuda")    # 1024-bit chunks
    short = torch.zeros((4, 64), dtype=torch.int32, device="cuda")
    idx = torch.zeros(4, dtype=torch.int32, device="cuda")
    for call in (lambda: ctx.encrypt_chunks(ks, narrow),
                 lambda: ctx.decrypt_chunks(ks, good, out=short),
                 lambda: ctx.decrypt_chunks(ks, good, key_idx=idx),
                 lambda: ctx.encrypt_blinded(ks, good, short),
                 lambda: ctx.decrypt_blinded(ks, good, good, out=narrow),
                 lambda: ctx.modexp_chunks_baseline(ks, narrow),
                 lambda: ctx.split(2048, torch.zeros(600, dtype=torch.uint8, device="cuda"), out=good),
                 lambda: ctx.join(2048, good, 1000, out=torch.zeros(999, dtype=torch.uint8, device="cuda")),
                 lambda: ctx.batch([(ks, good, short, P.pmkrsa.OP_ENCRYPT)])):
        with pytest.raises(ValueError):
            call()
    host_only = P.import_keyset_host(ks.export_blob())
    for call in (lambda: ctx.encrypt_chunks(host_only, good),
                 lambda: ctx.decrypt_chunks(host_only, good, use_crt=True),
                 lambda: ctx.encrypt_chunks(host_only, good[:0]),
                 lambda: ctx.autotune(host_only, 100, "decrypt", reps=1)):
        with pytest.raises(P.PMKError) as err:
            call()
        assert err.value.code == P.pmkrsa.PMK_EINVAL
    assert ctx.status() == 0
    host_only.free()
    ks.free()


def test_batched_workload_at_full_scale_against_the_oracle(env):
    """The batched workload at its stated size: 64 messages, sizes log-uniform
    over 4 KB - 25 MB, each with its own K in {2, 4, 8, 16} and width in
    {1024, 2048, 3072, 4096} bits, 70% full-d decryption, 10% CRT decryption,
    20% encryption.  The graph-replayed batch equals one call per job, and
    every job is checked against the oracle on 4 chunks including its last
    (the oracle computes with the library's exported keys)."""
    P, oracle, ctx = env
    from paper_2111_11924_gb300 import pmkrsa as B

    rng = np.random.default_rng(0x50444D4B0000C000)
    keysets, okeys, jobs = {}, {}, []
    for msg_i in range(64):
        size = int(np.exp(rng.uniform(np.log(4096), np.log(25e6))))
        K = int(rng.choice([2, 4, 8, 16]))
        nbits = int(rng.choice([1024, 2048, 3072, 4096]))
        op = int(rng.choice([B.OP_DECRYPT, B.OP_DECRYPT_CRT, B.OP_ENCRYPT], p=[0.7, 0.1, 0.2]))
        if (K, nbits) not in keysets:
            keysets[K, nbits] = ctx.keygen(K, nbits, 65537, 0x50444D4B0000C100 + 16 * K + nbits)
            okeys[K, nbits] = oracle.OracleKeys(K, nbits, 65537, keysets[K, nbits].export())
        ks = keysets[K, nbits]
        msg = torch.from_numpy(np.random.default_rng(msg_i).integers(0, 256, size, dtype=np.uint8)).cuda()
        plain = ctx.split(nbits, msg)
        src = plain if op == B.OP_ENCRYPT else ctx.encrypt_chunks(ks, plain)
        jobs.append((ks, src, torch.empty_like(src), op, okeys[K, nbits]))
    batch = ctx.batch([j[:4] for j in jobs])
    batch.launch()
    ctx.check()
    assert sum(j[1].shape[0] for j in jobs) > 250_000
    for ks, x, out, op, ok in jobs:
        ref = (ctx.encrypt_chunks(ks, x) if op == B.OP_ENCRYPT
               else ctx.decrypt_chunks(ks, x, use_crt=(op == B.OP_DECRYPT_CRT)))
        assert torch.equal(out, ref), (ks.nbits, ks.K, op, x.shape[0])
        n = x.shape[0]
        sample = np.unique(np.concatenate([rng.integers(0, n, 3), [n - 1]]))
        xin = x.cpu().numpy().view(np.uint32)[sample]
        want = (oracle.encrypt_chunks(xin, ok, threads=8, key_idx=sample % ok.K) if op == B.OP_ENCRYPT
                else oracle.decrypt_chunks(xin, ok, threads=8, key_idx=sample % ok.K))
        assert np.array_equal(out.cpu().numpy().view(np.uint32)[sample], want), (ks.nbits, ks.K, op, n)
    batch.destroy()
    for ks in keysets.values():
        ks.free()
