"""The whole-message calls on host buffers: error paths drain their stream,
and the context's stream-ordered staging is safe across streams and growth."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    import oracle
    import paper_2111_11924_gb300 as P

    ctx = P.Context(0)
    ks = ctx.keygen(4, 1024, 65537, 0x50444D4B00000A11)
    ok = oracle.keygen(4, 1024, 65537, 0x50444D4B00000A11)
    yield P, oracle, ctx, ks, ok
    ks.free()
    ctx.close()


def _msg(n, seed):
    return torch.from_numpy(np.random.default_rng(seed).integers(0, 256, n, dtype=np.uint8)).pin_memory()


def test_error_after_copy_returns_with_stream_idle(env, monkeypatch):
    P, oracle, ctx, ks, ok = env
    msg = _msg(2 << 20, 1)
    n = P.num_chunks(msg.numel(), ks.nbits)
    cipher = torch.empty((n, ks.limbs), dtype=torch.int32).pin_memory()
    back = torch.empty_like(msg).pin_memory()
    s = torch.cuda.Stream()
    ctx.encrypt_message_host(ks, msg, cipher, stream=s)
    monkeypatch.setenv("PMK_INJECT_FAULT", "after_copy")
    for call in (lambda: ctx.encrypt_message_host(ks, msg, cipher, stream=s),
                 lambda: ctx.decrypt_message_host(ks, cipher, back, stream=s)):
        with pytest.raises(P.PMKError) as err:
            call()
        assert err.value.code == P.pmkrsa.PMK_ECUDA
        assert s.query(), "a copy of the caller's buffer is still in flight"
    monkeypatch.delenv("PMK_INJECT_FAULT")
    ctx.decrypt_message_host(ks, cipher, back, stream=s)
    assert torch.equal(back, msg)


def test_staging_reused_and_grown_across_streams(env):
    """Alternate streams and grow the staging between calls; every result
    matches the oracle's ciphertext and round-trips."""
    P, oracle, ctx, ks, ok = env
    streams = [torch.cuda.Stream(), torch.cuda.Stream(), None]
    for i, size in enumerate((1000, 300_000, 5000, 2_000_000, 77)):
        msg = _msg(size, 10 + i)
        n = P.num_chunks(size, ks.nbits)
        cipher = torch.empty((n, ks.limbs), dtype=torch.int32).pin_memory()
        back = torch.empty_like(msg).pin_memory()
        s = streams[i % 3]
        ctx.encrypt_message_host(ks, msg, cipher, stream=s)
        ref = oracle.encrypt_chunks(oracle.split(msg.numpy(), ks.nbits)[:64], ok)
        assert np.array_equal(cipher.numpy().view(np.uint32)[:64], ref), size
        ctx.decrypt_message_host(ks, cipher, back, use_crt=bool(i % 2), stream=streams[(i + 1) % 3])
        assert torch.equal(back, msg), size
