"""Serving loop: requests admitted while others run overlap on the device,
and every result is bit-identical to the same request processed alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_each_result_same_alone_and_in_the_mix():
    import paper_2111_11924_gb300 as P
    from paper_2111_11924_gb300 import serving as SV

    ctx = P.Context(0)
    widths = (1024, 2048)
    keysets = {nb: ctx.keygen(4, nb, 65537, 0x50444D4B0000E000 + nb) for nb in widths}
    reqs = SV.poisson_requests(rate_per_s=20000, count=48, seed=11, widths=widths, min_bytes=100,
                               max_bytes=60_000)
    SV.prepare_payloads(ctx, keysets, reqs)
    server = SV.Server(ctx, keysets, budget_bytes=2_000_000, slots=8, use_crt=True)
    stats = server.serve(reqs)
    assert stats["status"] == 0
    assert stats["peak_in_flight"] > 1            # requests overlapped on the device
    assert stats["peak_device_bytes"] <= 2_000_000  # admission respected the budget
    mixed = [r.result.clone() for r in reqs]
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
    small = SV.Server(ctx, keysets, budget_bytes=biggest - 1, slots=8)
    for r in reqs:
        r.result = None
    with pytest.raises(ValueError):
        small.serve(reqs)
    ctx.close()


def test_corrupted_request_is_reported_and_isolated():
    """Fault injection from the host: one decryption request carries a chunk
    equal to its modulus.  The run reports PMK_ERANGE through the context's
    status, and every other request still gets its exact result."""
    import paper_2111_11924_gb300 as P
    from paper_2111_11924_gb300 import serving as SV

    ctx = P.Context(0)
    keysets = {1024: ctx.keygen(3, 1024, 65537, 0x50444D4B0000F100)}
    reqs = SV.poisson_requests(rate_per_s=20000, count=16, seed=9, widths=(1024,), p_decrypt=1.0, min_bytes=500,
                               max_bytes=20_000)
    SV.prepare_payloads(ctx, keysets, reqs)
    bad = reqs[5]
    N0 = keysets[1024].export()["N"][0]
    bad.payload[0] = torch.from_numpy(N0.view(np.int32).copy())  # chunk 0 (key 0) := N_0, out of range
    server = SV.Server(ctx, keysets, budget_bytes=10_000_000, slots=4, use_crt=True)
    stats = server.serve(reqs)
    assert stats["status"] == P.pmkrsa.PMK_ERANGE
    for r in reqs:
        if r is not bad:
            assert torch.equal(r.result, r.extra["message"]), r.rid
    assert ctx.status() == 0  # the status was read and cleared by the run
    ctx.close()
