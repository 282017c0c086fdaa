"""ctypes binding of libpmkrsa.so: one Python call per C-ABI entry point.

Device buffers are torch CUDA tensors (limb buffers as int32 tensors holding
uint32 bit patterns, messages as uint8 tensors); the CUDA stream is torch's
current stream on the context's device unless one is given.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import _native_build

PMK_OK, PMK_EINVAL, PMK_ERANGE, PMK_ENOMEM, PMK_ECUDA, PMK_EUNSUPPORTED, PMK_ETOOLARGE, PMK_ENOINV, PMK_EKEYINDEX = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)

_lib = None

OP_ENCRYPT, OP_DECRYPT, OP_DECRYPT_CRT = 0, 1, 2


class _Job(ctypes.Structure):
    """struct pmk_job of include/pmkrsa.h."""
    _fields_ = [("ks", ctypes.c_void_p), ("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p),
                ("n_chunks", ctypes.c_size_t), ("op", ctypes.c_int)]


class PMKError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else f"{strerror(code)} ({code})")


def load_library() -> ctypes.CDLL:
    """Load the in-tree native library; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _native_build.LIB
    if not os.path.exists(path):
        raise ImportError(f"native PMKRSA library not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P32 = ctypes.POINTER(ctypes.c_uint32)
    vp, u32, u64, sz, i = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t, ctypes.c_int
    sig = {
        "pmk_create": (i, [ctypes.POINTER(vp), i]),
        "pmk_destroy": (None, [vp]),
        "pmk_keygen": (i, [vp, u32, u32, u64, u64, ctypes.POINTER(vp)]),
        "pmk_keygen_host": (i, [u32, u32, u64, u64, P32, P32, P32, P32, P32, P32, P32]),
        "pmk_keyset_from_primes": (i, [vp, u32, u32, u64, P32, P32, ctypes.POINTER(vp)]),
        "pmk_keyset_export_fields": (i, [vp, P32, P32, P32, P32, P32, P32, P32]),
        "pmk_keygen_multiprime": (i, [vp, u32, u32, u32, u64, u64, ctypes.POINTER(vp)]),
        "pmk_keygen_host_multiprime": (i, [u32, u32, u32, u64, u64, P32, P32, P32, P32, P32]),
        "pmk_keyset_export_primes": (i, [vp, P32, P32, P32]),
        "pmk_keyset_from_primes_multi": (i, [vp, u32, u32, u32, u64, P32, ctypes.POINTER(vp)]),
        "pmk_keyset_export": (i, [vp, vp, ctypes.POINTER(sz)]),
        "pmk_keyset_import": (i, [vp, vp, sz, ctypes.POINTER(vp)]),
        "pmk_keyset_num_primes": (u32, [vp]),
        "pmk_keyset_num_keys": (u32, [vp]),
        "pmk_keyset_nbits": (u32, [vp]),
        "pmk_keyset_e": (u64, [vp]),
        "pmk_keyset_free": (None, [vp]),
        "pmk_payload_bytes": (sz, [u32]),
        "pmk_num_chunks": (sz, [sz, u32]),
        "pmk_split": (i, [vp, u32, vp, sz, vp, sz, vp]),
        "pmk_join": (i, [vp, u32, vp, sz, vp, sz, vp]),
        "pmk_encrypt_chunks": (i, [vp, vp, vp, vp, sz, vp, vp]),
        "pmk_decrypt_chunks": (i, [vp, vp, vp, vp, sz, vp, i, vp]),
        "pmk_modexp_chunks_baseline": (i, [vp, vp, vp, vp, sz, i, vp]),
        "pmk_encrypt_blinded": (i, [vp, vp, vp, vp, vp, vp, sz, vp]),
        "pmk_decrypt_blinded": (i, [vp, vp, vp, vp, vp, sz, i, vp]),
        "pmk_encrypt_message_host": (i, [vp, vp, vp, sz, vp, sz, vp]),
        "pmk_decrypt_message_host": (i, [vp, vp, vp, sz, vp, sz, i, vp]),
        "pmk_decrypt_message_host_noalloc": (i, [vp, vp, sz, vp, sz, i, vp]),
        "pmk_batch_create": (i, [vp, ctypes.POINTER(_Job), sz, ctypes.POINTER(vp)]),
        "pmk_batch_launch": (i, [vp, vp]),
        "pmk_batch_info": (i, [vp, ctypes.POINTER(sz), ctypes.POINTER(i)]),
        "pmk_set_batch_direct_max": (i, [vp, sz]),
        "pmk_batch_destroy": (None, [vp]),
        "pmk_sync_status": (i, [vp, vp]),
        "pmk_sync_status_detail": (i, [vp, vp, ctypes.POINTER(u64)]),
        "pmk_strerror": (ctypes.c_char_p, [i]),
        "pmk_measure_int_peak": (i, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(i)]),
        "pmk_measure_imad_peak": (i, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(i)]),
        "pmk_set_kernel_config": (i, [vp, u32, i, u32, u32]),
        "pmk_get_kernel_config": (i, [vp, u32, i, P32, P32]),
        "pmk_list_kernel_configs": (i, [u32, i, P32, P32, i]),
        "pmk_set_kernel_window": (i, [vp, u32, i, u32]),
        "pmk_get_kernel_window": (i, [vp, u32, i, P32]),
        "pmk_autotune": (i, [vp, vp, sz, i, i, P32, P32, ctypes.POINTER(ctypes.c_float)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load_library().pmk_strerror(code).decode()


def _check(rc: int, what: str) -> None:
    if rc != PMK_OK:
        raise PMKError(rc, what)


def payload_bytes(nbits: int) -> int:
    return int(load_library().pmk_payload_bytes(nbits))


def num_chunks(msg_len: int, nbits: int) -> int:
    return int(load_library().pmk_num_chunks(msg_len, nbits))


def _p32(a: np.ndarray):
    assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


_KEY_FIELDS = ("N", "d", "p", "q", "dp", "dq", "qinv")


def _key_arrays(K: int, nbits: int) -> dict:
    s, h = nbits // 32, nbits // 64
    return {f: np.zeros((K, s if f in ("N", "d") else h), np.uint32) for f in _KEY_FIELDS}


def keygen_host(K: int, nbits: int, e: int = 65537, seed: int = 0) -> dict:
    """Key initialisation on the host only (no GPU): dict of (K, limbs) uint32 arrays."""
    arrs = _key_arrays(K, nbits)
    _check(load_library().pmk_keygen_host(K, nbits, e, seed & (2**64 - 1), *[_p32(arrs[f]) for f in _KEY_FIELDS]),
           "pmk_keygen_host")
    return arrs


_MP_FIELDS = ("N", "d", "primes", "dexp", "coef")


def keygen_host_multiprime(K: int, nbits: int, nprimes: int, e: int = 65537, seed: int = 0) -> dict:
    """Multi-prime key initialisation on the host only: N, d, primes, dexp,
    coef as (K, nbits/32) uint32 arrays (the prime fields hold b values of
    nbits/(32 b) limbs each)."""
    arrs = {f: np.zeros((K, nbits // 32), np.uint32) for f in _MP_FIELDS}
    _check(load_library().pmk_keygen_host_multiprime(K, nbits, nprimes, e, seed & (2**64 - 1),
                                                     *[_p32(arrs[f]) for f in _MP_FIELDS]),
           "pmk_keygen_host_multiprime")
    return arrs


def _torch():
    import torch

    return torch


def chunk_shape(t, nbits: int, n_chunks=None, what: str = "chunks") -> int:
    """Check that a limb buffer has shape (n_chunks, nbits/32) (any n_chunks
    when None).  Returns its chunk count; raises ValueError otherwise, so
    that no call reads or writes past a buffer of another width or length."""
    if not isinstance(t, _torch().Tensor) or t.dim() != 2 or t.shape[1] != nbits // 32:
        raise ValueError(f"{what} must have shape (n_chunks, {nbits // 32}) for {nbits}-bit keys")
    if n_chunks is not None and t.shape[0] != n_chunks:
        raise ValueError(f"{what} holds {t.shape[0]} chunks, {n_chunks} expected")
    return int(t.shape[0])


def host_limb_buffer(t, nbits: int, what: str = "h_cipher"):
    """Check a host limb buffer for the *_host calls: a contiguous CPU int32
    (or uint32) tensor of shape (n_chunks, nbits/32).  Returns the chunk
    count; raises ValueError otherwise, before the library would read past it."""
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
        raise ValueError(f"{what} must be a CPU tensor")
    if t.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)) or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous int32 tensor")
    return chunk_shape(t, nbits, None, what)


def host_message_buffer(t, n_chunks: int, nbits: int, what: str = "h_msg"):
    """Check a host message buffer: a contiguous CPU uint8 tensor whose length
    gives exactly n_chunks chunks at this width.  Returns its length."""
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
        raise ValueError(f"{what} must be a CPU tensor")
    if t.dtype != torch.uint8 or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous uint8 tensor")
    P = nbits // 8 - 1
    if (t.numel() + P - 1) // P != n_chunks:
        raise ValueError(f"{what} of {t.numel()} bytes does not split into {n_chunks} chunks of {P} bytes")
    return int(t.numel())


class KeySet:
    """K key pairs resident on the context's device (pmk_keyset)."""

    def __init__(self, ctx: "Context", handle: ctypes.c_void_p):
        self._ctx = ctx
        self._h = handle
        lib = load_library()
        self.K = int(lib.pmk_keyset_num_keys(handle))
        self.nbits = int(lib.pmk_keyset_nbits(handle))
        self.e = int(lib.pmk_keyset_e(handle))
        self.nprimes = int(lib.pmk_keyset_num_primes(handle))
        self.limbs = self.nbits // 32

    @property
    def handle(self):
        if not self._h:
            raise ValueError("key set freed")
        return self._h

    def export(self) -> dict:
        """Key material as host arrays: N, d, p, q, dp, dq, qinv for a two-prime
        key set; N, d, primes, dexp, coef for a multi-prime one."""
        lib = load_library()
        if self.nprimes != 2:
            arrs = {f: np.zeros((self.K, self.limbs), np.uint32) for f in _MP_FIELDS}
            _check(lib.pmk_keyset_export_fields(self.handle, _p32(arrs["N"]), _p32(arrs["d"]), None, None, None, None, None),
                   "export")
            _check(lib.pmk_keyset_export_primes(self.handle, _p32(arrs["primes"]), _p32(arrs["dexp"]),
                                                _p32(arrs["coef"])), "export_primes")
            return arrs
        arrs = _key_arrays(self.K, self.nbits)
        _check(lib.pmk_keyset_export_fields(self.handle, *[_p32(arrs[f]) for f in _KEY_FIELDS]), "export")
        return arrs

    def export_blob(self) -> bytes:
        """The key set as a versioned little-endian blob (pmk_keyset_export)."""
        lib = load_library()
        n = ctypes.c_size_t(0)
        _check(lib.pmk_keyset_export(self.handle, None, ctypes.byref(n)), "pmk_keyset_export")
        buf = ctypes.create_string_buffer(n.value)
        _check(lib.pmk_keyset_export(self.handle, buf, ctypes.byref(n)), "pmk_keyset_export")
        return buf.raw[: n.value]

    def free(self) -> None:
        if self._h:
            load_library().pmk_keyset_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """A pmk_ctx bound to one CUDA device."""

    def __init__(self, device: int = 0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise PMKError(PMK_ECUDA, "no CUDA device: the PMKRSA path runs only on the GPU")
        self.device = int(device)
        torch.cuda.init()
        h = ctypes.c_void_p()
        _check(load_library().pmk_create(ctypes.byref(h), self.device), "pmk_create")
        self._h = h

    # ------------------------------------------------------------ plumbing
    @property
    def handle(self):
        if not self._h:
            raise ValueError("context closed")
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None):
            load_library().pmk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stream_handle(self, stream=None) -> int:
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return int(s.cuda_stream)

    def _dev(self, t, dtype, what):
        torch = _torch()
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.device.index != self.device:
            raise ValueError(f"{what} must be a CUDA tensor on device {self.device}")
        if t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"{what} must be a contiguous {dtype} tensor")
        return ctypes.c_void_p(t.data_ptr())

    def _limbs(self, t, nbits: int, n_chunks, what):
        """Device pointer of a chunk buffer: a contiguous int32 CUDA tensor on
        this device of shape (n_chunks, nbits/32)."""
        p = self._dev(t, _torch().int32, what)
        chunk_shape(t, nbits, n_chunks, what)
        return p

    def _bytes(self, t, n_bytes: int, what):
        """Device pointer of a contiguous uint8 CUDA tensor of n_bytes bytes."""
        p = self._dev(t, _torch().uint8, what)
        if t.numel() != n_bytes:
            raise ValueError(f"{what} holds {t.numel()} bytes, {n_bytes} expected")
        return p

    # ------------------------------------------------------------ keys
    def keygen(self, K: int, nbits: int, e: int = 65537, seed: int = 0, nprimes: int = 2) -> KeySet:
        """K key pairs; nprimes > 2 gives multi-prime keys (Section 2.1)."""
        h = ctypes.c_void_p()
        if nprimes == 2:
            _check(load_library().pmk_keygen(self.handle, K, nbits, e, seed & (2**64 - 1), ctypes.byref(h)),
                   "pmk_keygen")
        else:
            _check(load_library().pmk_keygen_multiprime(self.handle, K, nbits, nprimes, e, seed & (2**64 - 1),
                                                        ctypes.byref(h)), "pmk_keygen_multiprime")
        return KeySet(self, h)

    def import_keyset(self, blob: bytes) -> KeySet:
        """A key set restored from pmk_keyset_export's bytes, on this context's device."""
        h = ctypes.c_void_p()
        _check(load_library().pmk_keyset_import(self.handle, blob, len(blob), ctypes.byref(h)), "pmk_keyset_import")
        return KeySet(self, h)

    def keyset_from_primes(self, nbits: int, e: int, p: np.ndarray, q: np.ndarray) -> KeySet:
        p = np.ascontiguousarray(p, np.uint32)
        q = np.ascontiguousarray(q, np.uint32)
        K = p.shape[0]
        h = ctypes.c_void_p()
        _check(load_library().pmk_keyset_from_primes(self.handle, K, nbits, e, _p32(p), _p32(q), ctypes.byref(h)),
               "pmk_keyset_from_primes")
        return KeySet(self, h)

    def keyset_from_primes_multi(self, nbits: int, nprimes: int, e: int, primes: np.ndarray) -> KeySet:
        """Multi-prime key set from (K, nbits/32) limbs holding each key's nprimes primes."""
        primes = np.ascontiguousarray(primes, np.uint32)
        h = ctypes.c_void_p()
        _check(load_library().pmk_keyset_from_primes_multi(self.handle, primes.shape[0], nbits, nprimes, e,
                                                           _p32(primes), ctypes.byref(h)),
               "pmk_keyset_from_primes_multi")
        return KeySet(self, h)

    # ------------------------------------------------------------ hot path
    def split(self, nbits: int, msg, out=None, stream=None):
        torch = _torch()
        n = num_chunks(msg.numel(), nbits)
        if out is None:
            out = torch.empty((n, nbits // 32), dtype=torch.int32, device=msg.device)
        _check(load_library().pmk_split(self.handle, nbits, self._dev(msg, torch.uint8, "msg"), msg.numel(),
                                        self._limbs(out, nbits, n, "chunks"), n, self.stream_handle(stream)),
               "pmk_split")
        return out

    def join(self, nbits: int, chunks, msg_len: int, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty(msg_len, dtype=torch.uint8, device=chunks.device)
        _check(load_library().pmk_join(self.handle, nbits, self._limbs(chunks, nbits, None, "chunks"), chunks.shape[0],
                                       self._bytes(out, msg_len, "msg"), msg_len, self.stream_handle(stream)),
               "pmk_join")
        return out

    def _key_idx(self, key_idx, n: int):
        """Device pointer of an explicit key-index vector (int32 CUDA tensor of n), or None."""
        if key_idx is None:
            return None
        p = self._dev(key_idx, _torch().int32, "key_idx")
        if key_idx.numel() != n:
            raise ValueError(f"key_idx must hold one key index per chunk ({n})")
        return p

    def encrypt_chunks(self, ks: KeySet, chunks, out=None, stream=None, key_idx=None):
        """c[t] = m[t]^e mod N_k with k = t mod K, or k = key_idx[t] when given."""
        torch = _torch()
        if out is None:
            out = torch.empty_like(chunks)
        n = chunk_shape(chunks, ks.nbits, None, "in")
        _check(load_library().pmk_encrypt_chunks(self.handle, ks.handle, self._limbs(chunks, ks.nbits, n, "in"),
                                                 self._limbs(out, ks.nbits, n, "out"), n,
                                                 self._key_idx(key_idx, chunks.shape[0]),
                                                 self.stream_handle(stream)), "pmk_encrypt_chunks")
        return out

    def decrypt_chunks(self, ks: KeySet, chunks, use_crt: bool = False, out=None, stream=None, key_idx=None):
        """m[t] = c[t]^d mod N_k with k = t mod K, or k = key_idx[t] when given."""
        torch = _torch()
        if out is None:
            out = torch.empty_like(chunks)
        n = chunk_shape(chunks, ks.nbits, None, "in")
        _check(load_library().pmk_decrypt_chunks(self.handle, ks.handle, self._limbs(chunks, ks.nbits, n, "in"),
                                                 self._limbs(out, ks.nbits, n, "out"), n,
                                                 self._key_idx(key_idx, chunks.shape[0]), int(use_crt),
                                                 self.stream_handle(stream)), "pmk_decrypt_chunks")
        return out

    def modexp_chunks_baseline(self, ks: KeySet, chunks, decrypt: bool = True, out=None, stream=None):
        """The plain thread-per-chunk, binary-exponent kernel (a measured baseline)."""
        torch = _torch()
        out = torch.empty_like(chunks) if out is None else out
        n = chunk_shape(chunks, ks.nbits, None, "in")
        _check(load_library().pmk_modexp_chunks_baseline(self.handle, ks.handle, self._limbs(chunks, ks.nbits, n, "in"),
                                                         self._limbs(out, ks.nbits, n, "out"), n,
                                                         int(decrypt), self.stream_handle(stream)),
               "pmk_modexp_chunks_baseline")
        return out

    def encrypt_blinded(self, ks: KeySet, chunks, rnd, out_cstar=None, out_cr=None, stream=None):
        """Algorithm 1 encryption with the random matrix R: returns (C*, C_R)."""
        torch = _torch()
        out_cstar = torch.empty_like(chunks) if out_cstar is None else out_cstar
        out_cr = torch.empty_like(chunks) if out_cr is None else out_cr
        n = chunk_shape(chunks, ks.nbits, None, "m")
        _check(load_library().pmk_encrypt_blinded(self.handle, ks.handle, self._limbs(chunks, ks.nbits, n, "m"),
                                                  self._limbs(rnd, ks.nbits, n, "r"),
                                                  self._limbs(out_cstar, ks.nbits, n, "cstar"),
                                                  self._limbs(out_cr, ks.nbits, n, "cr"), n,
                                                  self.stream_handle(stream)), "pmk_encrypt_blinded")
        return out_cstar, out_cr

    def decrypt_blinded(self, ks: KeySet, cstar, cr, use_crt: bool = False, out=None, stream=None):
        """Algorithm 1 decryption with R: m = (c* c_r^-1)^d mod N."""
        torch = _torch()
        out = torch.empty_like(cstar) if out is None else out
        n = chunk_shape(cstar, ks.nbits, None, "cstar")
        _check(load_library().pmk_decrypt_blinded(self.handle, ks.handle, self._limbs(cstar, ks.nbits, n, "cstar"),
                                                  self._limbs(cr, ks.nbits, n, "cr"), self._limbs(out, ks.nbits, n, "m"),
                                                  n, int(use_crt), self.stream_handle(stream)),
               "pmk_decrypt_blinded")
        return out

    def encrypt_message_host(self, ks: KeySet, h_msg, h_cipher, stream=None) -> None:
        """Host buffers (torch CPU tensors, ideally pinned): uint8 message -> int32 limb buffer."""
        n = host_limb_buffer(h_cipher, ks.nbits)
        L = host_message_buffer(h_msg, n, ks.nbits)
        _check(load_library().pmk_encrypt_message_host(self.handle, ks.handle, ctypes.c_void_p(h_msg.data_ptr()),
                                                       L, ctypes.c_void_p(h_cipher.data_ptr()), n,
                                                       self.stream_handle(stream)), "pmk_encrypt_message_host")

    def decrypt_message_host(self, ks: KeySet, h_cipher, h_msg, use_crt: bool = False, stream=None) -> None:
        n = host_limb_buffer(h_cipher, ks.nbits)
        L = host_message_buffer(h_msg, n, ks.nbits)
        _check(load_library().pmk_decrypt_message_host(self.handle, ks.handle, ctypes.c_void_p(h_cipher.data_ptr()), n,
                                                       ctypes.c_void_p(h_msg.data_ptr()), L, int(use_crt),
                                                       self.stream_handle(stream)), "pmk_decrypt_message_host")

    def batch(self, jobs) -> "Batch":
        """Plan and capture a batch: jobs = [(keyset, in_tensor, out_tensor, op), ...]
        with op one of OP_ENCRYPT, OP_DECRYPT, OP_DECRYPT_CRT."""
        torch = _torch()
        arr = (_Job * max(1, len(jobs)))()
        for k, (ks, t_in, t_out, op) in enumerate(jobs):
            n = chunk_shape(t_in, ks.nbits, None, "in")
            arr[k] = _Job(ks.handle, self._limbs(t_in, ks.nbits, n, "in").value,
                          self._limbs(t_out, ks.nbits, n, "out").value, n, int(op))
        h = ctypes.c_void_p()
        _check(load_library().pmk_batch_create(self.handle, arr, len(jobs), ctypes.byref(h)), "pmk_batch_create")
        return Batch(self, h, jobs)

    def set_batch_direct_max(self, max_jobs: int) -> None:
        """pmk_set_batch_direct_max: batches planned from now on with at most
        max_jobs jobs run every job as its own grid launch (default 256);
        0 sends every job below one GPU-full through the persistent queues."""
        _check(load_library().pmk_set_batch_direct_max(self.handle, int(max_jobs)), "pmk_set_batch_direct_max")

    def status(self, stream=None) -> int:
        """Synchronise and return (and clear) the device-side error code."""
        return int(load_library().pmk_sync_status(self.handle, self.stream_handle(stream)))

    def status_detail(self, stream=None) -> tuple:
        """(code, first failing chunk or None): pmk_sync_status_detail."""
        first = ctypes.c_uint64(0)
        code = int(load_library().pmk_sync_status_detail(self.handle, self.stream_handle(stream), ctypes.byref(first)))
        return code, (None if first.value == 2**64 - 1 else int(first.value))

    def check(self, stream=None) -> None:
        _check(self.status(stream), "device status")

    # ------------------------------------------------------------ tuning / measurement
    def measure_int_peak(self) -> dict:
        m, mhz, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        _check(load_library().pmk_measure_int_peak(self.handle, ctypes.byref(m), ctypes.byref(mhz), ctypes.byref(sms)),
               "pmk_measure_int_peak")
        return {"macs_per_clk_per_sm": m.value, "sm_mhz": mhz.value, "num_sms": sms.value}

    def measure_imad_peak(self) -> dict:
        """The INT32 multiply-add (mad.lo) issue rate per clock per SM, measured on this GPU."""
        m, mhz, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        _check(load_library().pmk_measure_imad_peak(self.handle, ctypes.byref(m), ctypes.byref(mhz),
                                                    ctypes.byref(sms)), "pmk_measure_imad_peak")
        return {"mad_lo_per_clk_per_sm": m.value, "sm_mhz": mhz.value, "num_sms": sms.value}

    def set_kernel_config(self, limbs: int, crt: bool, tpi: int, form: int = 0) -> None:
        """Lanes per instance and Montgomery form for (limbs, crt); tpi = 0 restores the default."""
        _check(load_library().pmk_set_kernel_config(self.handle, limbs, int(crt), tpi, form), "pmk_set_kernel_config")

    def set_kernel_window(self, limbs: int, crt: bool, max_window: int) -> None:
        """Widest exponent window for (limbs, crt): 5 (16 odd powers per
        exponentiation in shared memory), 4 (8 odd powers, more resident
        exponentiations per SM) or 0 for the default (5)."""
        _check(load_library().pmk_set_kernel_window(self.handle, limbs, int(crt), max_window),
               "pmk_set_kernel_window")

    def get_kernel_window(self, limbs: int, crt: bool) -> int:
        w = np.zeros(1, np.uint32)
        _check(load_library().pmk_get_kernel_window(self.handle, limbs, int(crt), _p32(w)), "pmk_get_kernel_window")
        return int(w[0])

    def autotune(self, ks: KeySet, n_chunks: int, mode: str = "decrypt", reps: int = 3,
                 cache: "TuneCache | None" = None) -> dict:
        """Time every compiled geometry, with each window bound (5 and 4), for
        this key set and batch size; keep the fastest.  mode: "encrypt",
        "decrypt" (full d) or "crt".  With a TuneCache, a result stored for
        this GPU, width, prime count, mode and batch-size bucket is applied
        without timing, and a new result is stored."""
        m = {"encrypt": 0, "decrypt": 1, "crt": 2}[mode]
        limbs = ks.nbits // 32 // (ks.nprimes if mode == "crt" else 1)
        key = None
        if cache is not None:
            key = cache.key(_torch().cuda.get_device_name(self.device), ks.nbits, ks.nprimes, mode, n_chunks)
            hit = cache.get(key)
            if hit is not None:
                self.set_kernel_config(limbs, mode == "crt", hit["tpi"], hit["form"])
                self.set_kernel_window(limbs, mode == "crt", hit["window"])
                return dict(hit) | {"cached": True}
        tpi, form, ms = np.zeros(1, np.uint32), np.zeros(1, np.uint32), ctypes.c_float()
        _check(load_library().pmk_autotune(self.handle, ks.handle, n_chunks, m, reps, _p32(tpi), _p32(form),
                                           ctypes.byref(ms)), "pmk_autotune")
        res = {"tpi": int(tpi[0]), "form": int(form[0]), "window": self.get_kernel_window(limbs, mode == "crt"),
               "ms": ms.value}
        if cache is not None:
            cache.put(key, res)
        return res

    def copy_kernel_configs_from(self, other: "Context", keysets: dict) -> None:
        """Take other's kernel geometry and window bound for every limb count
        the key sets use (full width and CRT residues)."""
        for ks in keysets.values():
            for limbs, crt in ((ks.nbits // 32, False), (ks.nbits // 32 // ks.nprimes, True)):
                tpi, form = other.get_kernel_config(limbs, crt)
                self.set_kernel_config(limbs, crt, tpi, form)
                self.set_kernel_window(limbs, crt, other.get_kernel_window(limbs, crt))

    def get_kernel_config(self, limbs: int, crt: bool) -> tuple:
        tpi, form = np.zeros(1, np.uint32), np.zeros(1, np.uint32)
        _check(load_library().pmk_get_kernel_config(self.handle, limbs, int(crt), _p32(tpi), _p32(form)),
               "pmk_get_kernel_config")
        return int(tpi[0]), int(form[0])


class TuneCache:
    """Autotuner results persisted as JSON, keyed by GPU name, key width,
    prime count, mode and batch size rounded up to a power of two (the best
    geometry depends on how many exponentiations fill the GPU)."""

    def __init__(self, path: str):
        import json
        import os

        self.path = path
        self._json, self._os = json, os
        try:
            with open(path) as f:
                self.entries = json.load(f)
        except (OSError, ValueError):
            self.entries = {}

    @staticmethod
    def key(gpu: str, nbits: int, nprimes: int, mode: str, n_chunks: int) -> str:
        bucket = 1 << max(0, (int(n_chunks) - 1).bit_length())
        return f"{gpu}|{nbits}|{nprimes}|{mode}|{bucket}"

    def get(self, key: str):
        e = self.entries.get(key)
        if e is None:
            return None
        return {"tpi": int(e["tpi"]), "form": int(e["form"]), "window": int(e.get("window", 5)), "ms": float(e["ms"])}

    def put(self, key: str, res: dict) -> None:
        self.entries[key] = {"tpi": int(res["tpi"]), "form": int(res["form"]), "window": int(res.get("window", 5)),
                             "ms": float(res["ms"])}
        tmp = f"{self.path}.tmp{self._os.getpid()}"
        with open(tmp, "w") as f:
            self._json.dump(self.entries, f, indent=1, sort_keys=True)
        self._os.replace(tmp, self.path)


def kernel_configs(limbs: int, crt: bool) -> list:
    """Compiled (tpi, form) geometries for an exponentiation over `limbs` limbs."""
    lib = load_library()
    n = lib.pmk_list_kernel_configs(limbs, int(crt), None, None, 0)
    if n <= 0:
        return []
    tpi, form = np.zeros(n, np.uint32), np.zeros(n, np.uint32)
    lib.pmk_list_kernel_configs(limbs, int(crt), _p32(tpi), _p32(form), n)
    return list(zip(tpi.tolist(), form.tolist()))


def import_keyset_host(blob: bytes) -> KeySet:
    """A host-only key set from a blob (pmk_keyset_import with no context):
    it can be exported and inspected but not used by device calls."""
    h = ctypes.c_void_p()
    _check(load_library().pmk_keyset_import(None, blob, len(blob), ctypes.byref(h)), "pmk_keyset_import")
    return KeySet(None, h)


def decrypt_message_host_noalloc(ks: KeySet, h_cipher, h_msg, use_crt: bool = False, stream=None) -> int:
    """pmk_decrypt_message_host_noalloc: decrypt without any device allocation
    (device staging in the library's fixed array).  Returns the PMK_* code."""
    torch = _torch()
    n = host_limb_buffer(h_cipher, ks.nbits)
    L = host_message_buffer(h_msg, n, ks.nbits)
    if stream is not None:
        s = int(stream.cuda_stream)
    elif ks._ctx is not None:
        s = int(torch.cuda.current_stream(ks._ctx.device).cuda_stream)
    else:
        s = 0  # a host-only key set: the library refuses it before any device work
    return int(load_library().pmk_decrypt_message_host_noalloc(
        ks.handle, ctypes.c_void_p(h_cipher.data_ptr()), n, ctypes.c_void_p(h_msg.data_ptr()),
        L, int(use_crt), ctypes.c_void_p(s)))


class Batch:
    """A planned, graph-captured batch (pmk_batch); keeps its job tensors alive."""

    def __init__(self, ctx: Context, handle, jobs):
        self._ctx, self._h, self._jobs = ctx, handle, list(jobs)
        n, k = ctypes.c_size_t(), ctypes.c_int()
        _check(load_library().pmk_batch_info(handle, ctypes.byref(n), ctypes.byref(k)), "pmk_batch_info")
        self.n_tasks, self.n_kernels = n.value, k.value

    def launch(self, stream=None) -> None:
        _check(load_library().pmk_batch_launch(self._h, ctypes.c_void_p(self._ctx.stream_handle(stream))),
               "pmk_batch_launch")

    def destroy(self) -> None:
        if self._h:
            load_library().pmk_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
