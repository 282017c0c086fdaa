"""Serving loop: requests admitted while others run are coalesced into
batches that overlap on the device; every result is bit-identical to the same
request processed alone and to the oracle; each request gets its own status."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _oracle_check_encrypt(oracle, okeys, r, sample=6):
    """A sample of an encryption request's ciphertext (first, last and random
    chunks) against the oracle's c_t = m_t^e mod N_{t mod K}."""
    nbits = r.nbits
    m = oracle.split(r.extra["message"].numpy(), nbits)
    n = m.shape[0]
    rng = np.random.default_rng(r.rid)
    idx = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, sample)]))
    ok = okeys[nbits]
    want = oracle.encrypt_chunks(m[idx], ok, key_idx=idx % ok.K)
    got = r.result.numpy().view(np.uint32)[idx]
    assert np.array_equal(got, want), (r.rid, idx)


def _serve_and_check(widths, count, seed, max_bytes, lanes, budget, oracle_keygen=True):
    """oracle_keygen: the oracle generates its own keys and they must equal
    the library's; otherwise (wide keys, where the oracle's keygen takes
    minutes) the oracle computes with the library's exported key material."""
    import oracle
    import paper_2111_11924_gb300 as P
    from paper_2111_11924_gb300 import serving as SV

    ctx = P.Context(0)
    K = 4
    keysets = {nb: ctx.keygen(K, nb, 65537, 0x50444D4B0000E000 + nb) for nb in widths}
    okeys = {}
    for nb in widths:
        ex = keysets[nb].export()
        if oracle_keygen:
            okeys[nb] = oracle.keygen(K, nb, 65537, 0x50444D4B0000E000 + nb)
            assert all(np.array_equal(ex[f], okeys[nb].a[f]) for f in okeys[nb].a)
        else:
            okeys[nb] = oracle.OracleKeys(K, nb, 65537, ex)
    reqs = SV.poisson_requests(rate_per_s=20000, count=count, seed=seed, widths=widths, min_bytes=100,
                               max_bytes=max_bytes)
    SV.prepare_payloads(ctx, keysets, reqs)
    server = SV.Server(ctx, keysets, budget_bytes=budget, slots=32, use_crt=True, lanes=lanes)
    stats = server.serve(reqs)
    assert stats["status"] == 0 and stats["failed_requests"] == []
    assert stats["peak_in_flight"] > 1                # requests overlapped
    assert stats["batches"] < len(reqs)               # and were coalesced
    assert stats["peak_device_bytes"] <= budget       # admission respected the budget
    mixed = [r.result.clone() for r in reqs]
    for r in reqs:
        if r.op == "encrypt":
            _oracle_check_encrypt(oracle, okeys, r)
    # every request again, alone, through the plain per-call path
    for r in reqs:
        r.result = None
    alone_stats = server.serve_one_at_a_time(reqs)
    assert alone_stats["status"] == 0
    for r, m in zip(reqs, mixed):
        assert torch.equal(r.result, m), r.rid
        if r.op == "decrypt":
            assert torch.equal(m, r.extra["message"]), r.rid
        else:
            ks = keysets[r.nbits]
            back = ctx.join(r.nbits, ctx.decrypt_chunks(ks, m.cuda()), r.msg_len)
            assert torch.equal(back.cpu(), r.extra["message"]), r.rid
    server.close()
    ctx.close()


def test_each_result_same_alone_and_in_the_mix():
    _serve_and_check((1024, 2048), count=48, seed=11, max_bytes=60_000, lanes=4, budget=2_000_000)


def test_serving_widths_of_the_serving_workload():
    """The serving workload's key widths, 2048, 3072 and 4096 bits."""
    _serve_and_check((2048, 3072, 4096), count=36, seed=12, max_bytes=200_000, lanes=3, budget=8_000_000,
                     oracle_keygen=False)


def test_per_request_streams_without_packing():
    """The loop with coalescing off (each request on its own stream) gives the
    same results as one request at a time."""
    import paper_2111_11924_gb300 as P
    from paper_2111_11924_gb300 import serving as SV

    ctx = P.Context(0)
    keysets = {1024: ctx.keygen(3, 1024, 65537, 0x50444D4B0000E600)}
    reqs = SV.poisson_requests(rate_per_s=20000, count=20, seed=13, widths=(1024,), min_bytes=100, max_bytes=30_000)
    SV.prepare_payloads(ctx, keysets, reqs)
    server = SV.Server(ctx, keysets, budget_bytes=5_000_000, slots=8)
    stats = server.serve(reqs, coalesce=False)
    assert stats["status"] == 0
    for r in reqs:
        if r.op == "decrypt":
            assert torch.equal(r.result, r.extra["message"]), r.rid
    server.close()
    ctx.close()


def test_budget_admission_serialises_and_rejects():
    """A budget that fits one request at a time admits them one by one
    (never two in flight) and still produces every result; a request larger
    than the whole budget is refused before anything runs."""
    import paper_2111_11924_gb300 as P
    from paper_2111_11924_gb300 import serving as SV

    ctx = P.Context(0)
    keysets = {1024: ctx.keygen(2, 1024, 65537, 0x50444D4B0000EF00)}
    reqs = SV.poisson_requests(rate_per_s=50000, count=12, seed=5, widths=(1024,), min_bytes=20_000,
                               max_bytes=30_000)
    SV.prepare_payloads(ctx, keysets, reqs)
    biggest = max(r.device_bytes() for r in reqs)
    server = SV.Server(ctx, keysets, budget_bytes=biggest + 1, slots=8, use_crt=False)
    stats = server.serve(reqs)
    assert stats["status"] == 0 and stats["peak_in_flight"] == 1 and stats["peak_device_bytes"] <= biggest + 1
    for r in reqs:
        if r.op == "decrypt":
            assert torch.equal(r.result, r.extra["message"]), r.rid
    server.close()
    small = SV.Server(ctx, keysets, budget_bytes=biggest - 1, slots=8)
    for r in reqs:
        r.result = None
    with pytest.raises(ValueError):
        small.serve(reqs)
    small.close()
    ctx.close()


def test_corrupted_request_is_reported_and_isolated():
    """Fault injection from the host: two decryption requests carry a chunk
    equal to its modulus.  Exactly those two requests report PMK_ERANGE, by
    their own status, and every other request, batched with them or not,
    still gets its exact result."""
    import paper_2111_11924_gb300 as P
    from paper_2111_11924_gb300 import serving as SV

    ctx = P.Context(0)
    keysets = {1024: ctx.keygen(3, 1024, 65537, 0x50444D4B0000F100)}
    reqs = SV.poisson_requests(rate_per_s=20000, count=16, seed=9, widths=(1024,), p_decrypt=1.0, min_bytes=500,
                               max_bytes=20_000)
    SV.prepare_payloads(ctx, keysets, reqs)
    N = keysets[1024].export()["N"]
    bad = [reqs[5], reqs[11]]
    bad[0].payload[0] = torch.from_numpy(N[0].view(np.int32).copy())  # chunk 0 (key 0) := N_0, out of range
    t = bad[1].payload.shape[0] - 1
    bad[1].payload[t] = torch.from_numpy(N[t % 3].view(np.int32).copy())  # its last chunk := its key's modulus
    server = SV.Server(ctx, keysets, budget_bytes=10_000_000, slots=16, use_crt=True, lanes=2)
    stats = server.serve(reqs)
    assert stats["status"] == P.pmkrsa.PMK_ERANGE
    assert sorted(stats["failed_requests"]) == sorted(r.rid for r in bad)
    for r in reqs:
        if r not in bad:
            assert r.status == 0 and torch.equal(r.result, r.extra["message"]), r.rid
        else:
            assert r.status == P.pmkrsa.PMK_ERANGE
    assert ctx.status() == 0
    server.close()
    ctx.close()
