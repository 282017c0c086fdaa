"""The allocation-free decryption entry point against the allocating one.

pmk_decrypt_message_host_noalloc is for callers that cannot let the library
call cudaMalloc (device memory handed to another allocator under a fixed
budget, or a latency-critical path): it stages its device data in one fixed
array built into the library.  Its output must equal pmk_decrypt_message_host's
bit for bit, call after call, although the array keeps the previous call's
contents.  This file is collected last, so a failure here cannot hide the
results of the other test files.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    import paper_2111_11924_gb300 as P
    from paper_2111_11924_gb300 import workloads as W

    ctx = P.Context(0)
    w = W.FILE_1MIB_2048
    ks = ctx.keygen(w.K, w.nbits, w.e, w.key_seed)
    yield P, ctx, ks, w
    ks.free()
    ctx.close()


def _cipher_of(ctx, ks, msg):
    import paper_2111_11924_gb300 as P

    n = P.num_chunks(msg.numel(), ks.nbits)
    cipher = torch.empty((n, ks.nbits // 32), dtype=torch.int32).pin_memory()
    ctx.encrypt_message_host(ks, msg, cipher)
    return cipher


def test_noalloc_equals_allocating_call_twice(setup):
    P, ctx, ks, w = setup
    lib = P.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(2024)
    # two calls in a row on each of two messages of different sizes (the second smaller)
    for length in (w.msg_bytes, 70001):
        msg = torch.from_numpy(rng.integers(0, 256, length, dtype=np.uint8)).pin_memory()
        cipher = _cipher_of(ctx, ks, msg)
        n = cipher.shape[0]
        for use_crt in (0, 1):
            ref = torch.zeros(length, dtype=torch.uint8).pin_memory()
            ctx.decrypt_message_host(ks, cipher, ref, use_crt=bool(use_crt))
            for call in range(2):
                out = torch.full((length,), 0xA5, dtype=torch.uint8).pin_memory()
                rc = lib.pmk_decrypt_message_host_noalloc(ks.handle, ctypes.c_void_p(cipher.data_ptr()), n,
                                                          ctypes.c_void_p(out.data_ptr()), length, use_crt, stream)
                assert rc == P.pmkrsa.PMK_OK, (length, use_crt, call, P.strerror(rc))
                assert torch.equal(out, ref), (length, use_crt, call)
        assert torch.equal(ref, msg)


def test_noalloc_reports_range_error_then_recovers(setup):
    P, ctx, ks, w = setup
    msg = torch.from_numpy(np.random.default_rng(5).integers(0, 256, 5000, dtype=np.uint8)).pin_memory()
    cipher = _cipher_of(ctx, ks, msg)
    bad = cipher.clone().pin_memory()
    N = ks.export()["N"]
    bad[3] = torch.from_numpy(N[3 % ks.K].view(np.int32).copy())  # chunk 3 := N_3, not below its modulus
    out = torch.empty_like(msg).pin_memory()
    assert P.pmkrsa.decrypt_message_host_noalloc(ks, bad, out) == P.pmkrsa.PMK_ERANGE
    # the status word is cleared by the next call
    assert P.pmkrsa.decrypt_message_host_noalloc(ks, cipher, out) == P.pmkrsa.PMK_OK
    assert torch.equal(out, msg)


def test_noalloc_rejects_requests_beyond_its_capacity(setup):
    P, ctx, ks, w = setup
    length = 40 << 20  # 40 MiB of message does not fit the 32 MiB array
    n = P.num_chunks(length, ks.nbits)
    cipher = np.zeros((n, ks.nbits // 32), np.uint32)
    out = np.zeros(length, np.uint8)
    rc = P.load_library().pmk_decrypt_message_host_noalloc(ks.handle, ctypes.c_void_p(cipher.ctypes.data), n,
                                                           ctypes.c_void_p(out.ctypes.data), length, 0, None)
    assert rc == P.pmkrsa.PMK_ETOOLARGE
    assert "capacity" in P.strerror(rc)


def test_noalloc_multiprime_key_set(setup):
    """The allocation-free call on a 3-prime key set (CRT over three primes)
    equals the allocating call and recovers the message."""
    P, ctx, _, _ = setup
    ks = ctx.keygen(4, 3072, 65537, 0x50444D4B0000EA00, nprimes=3)
    msg = torch.from_numpy(np.random.default_rng(8).integers(0, 256, 200_003, dtype=np.uint8)).pin_memory()
    cipher = _cipher_of(ctx, ks, msg)
    for use_crt in (False, True):
        ref = torch.zeros_like(msg).pin_memory()
        ctx.decrypt_message_host(ks, cipher, ref, use_crt=use_crt)
        out = torch.full_like(msg, 0x5A).pin_memory()
        assert P.pmkrsa.decrypt_message_host_noalloc(ks, cipher, out, use_crt=use_crt) == P.pmkrsa.PMK_OK
        assert torch.equal(out, ref) and torch.equal(out, msg), use_crt
    ks.free()


def test_noalloc_empty_call_only_sets_up(setup):
    """A call with no chunks performs only the one-time set-up (the array's
    device address), so a caller can commit the array early in a process."""
    P, ctx, ks, w = setup
    lib = P.load_library()
    assert lib.pmk_decrypt_message_host_noalloc(ks.handle, None, 0, None, 0, 0, None) == P.pmkrsa.PMK_OK


def test_noalloc_rejects_chunk_counts_beyond_the_bound(setup):
    """2^32 chunks or more are refused before any size arithmetic, even when
    (msg_len, n_chunks) agree with each other."""
    P, ctx, ks, w = setup
    lib = P.load_library()
    payload = P.payload_bytes(ks.nbits)
    length = (1 << 32) * payload  # exactly 2^32 chunks
    n = P.num_chunks(length, ks.nbits)
    assert n == 1 << 32
    dummy = np.zeros(16, np.uint32)
    rc = lib.pmk_decrypt_message_host_noalloc(ks.handle, ctypes.c_void_p(dummy.ctypes.data), n,
                                              ctypes.c_void_p(dummy.ctypes.data), length, 0, None)
    assert rc == P.pmkrsa.PMK_EINVAL


def test_noalloc_error_after_copy_leaves_stream_idle(setup, monkeypatch):
    """A failure injected on the host right after the ciphertext copy is
    queued: the call reports it and returns with its stream idle; the next
    call is unaffected."""
    P, ctx, ks, w = setup
    msg = torch.from_numpy(np.random.default_rng(9).integers(0, 256, 3 << 20, dtype=np.uint8)).pin_memory()
    cipher = _cipher_of(ctx, ks, msg)
    out = torch.zeros_like(msg).pin_memory()
    stream = torch.cuda.Stream()
    monkeypatch.setenv("PMK_INJECT_FAULT", "after_copy")
    assert P.pmkrsa.decrypt_message_host_noalloc(ks, cipher, out, stream=stream) == P.pmkrsa.PMK_ECUDA
    assert stream.query(), "work left in flight on the caller's stream"
    monkeypatch.delenv("PMK_INJECT_FAULT")
    assert P.pmkrsa.decrypt_message_host_noalloc(ks, cipher, out, stream=stream) == P.pmkrsa.PMK_OK
    assert torch.equal(out, msg)
