"""PMKRSA oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow CPU restatement of what the PMKRSA hot path computes
("A Variant RSA Acceleration with Parallelization", arXiv 2111.11924).
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` leg / ``--impl reference`` arm may import it; the product
package never does, and this module never imports the product.

What lives where:
  * ``pmk_oracle.c`` -- schoolbook bignum (Knuth Algorithm D division),
    Algorithm 2 square-and-multiply, the Garner form of the Section 2.1 CRT
    equations and its multi-prime extension, extended Euclid, the seeded key
    initialisation of Algorithm 1 (two primes or b primes), and Algorithm 1's blinded encryption / decryption with the
    random matrix R (see that file's header for the readings it fixes).
  * this file -- ctypes marshalling, plus ``split``/``join`` written
    directly from their definitions (Section 3.1: the message is cut into
    chunks, each read as a little-endian integer; chunk t belongs to key
    t mod K, i.e. the i x j reshape fills column by column with one row per
    key).

Every function here is pinned in ``tests/test_oracle.py`` against things
other than itself: the textbook 3233 example, brute force over tiny
moduli, Python's own ``pow``/``divmod``, sympy's primality test and the
RSA / PMKRSA round-trip identities.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pmk_oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain C99, no architecture flags)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(ctypes.c_uint32)
            i = ctypes.c_int
            lib.oracle_mulmod.argtypes = [P, P, P, i, P]
            lib.oracle_divmod.argtypes = [P, i, P, i, P, i, P, i]
            lib.oracle_modexp.argtypes = [P, i, P, i, P, i, P]
            lib.oracle_crt.argtypes = [P, P, P, P, P, P, i, P]
            lib.oracle_modinv.argtypes = [P, P, i, P]
            lib.oracle_keygen.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                          P, P, P, P, P, P, P]
            lib.oracle_modexp_chunks.argtypes = [P, P, i, P, i, P, i, ctypes.c_long, ctypes.c_long]
            lib.oracle_crt_chunks.argtypes = [P, P, i, P, P, P, P, P, i, ctypes.c_long, ctypes.c_long]
            lib.oracle_keygen_mp.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                             ctypes.c_uint64, P, P, P, P, P]
            lib.oracle_crt_mp.argtypes = [P, i, i, P, P, P, P]
            lib.oracle_crt_mp_chunks.argtypes = [P, P, i, i, P, P, P, i, ctypes.c_long, ctypes.c_long]
            lib.oracle_blind_encrypt_chunks.argtypes = [P, P, P, P, i, P, i, P, i, ctypes.c_long, ctypes.c_long]
            lib.oracle_blind_decrypt_chunks.argtypes = [P, P, P, i, P, i, P, i, ctypes.c_long, ctypes.c_long]
            _lib = lib
    return _lib


# ---------------------------------------------------------------- limbs

def to_limbs(x: int, n: int) -> np.ndarray:
    """Non-negative int -> n little-endian uint32 limbs."""
    if x < 0 or x.bit_length() > 32 * n:
        raise ValueError("value does not fit")
    return np.frombuffer(x.to_bytes(4 * n, "little"), dtype="<u4").astype(np.uint32)


def from_limbs(a) -> int:
    return int.from_bytes(np.ascontiguousarray(a, dtype="<u4").tobytes(), "little")


def _ptr(a: np.ndarray):
    assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _nlimbs(*xs: int) -> int:
    return max(1, max((x.bit_length() + 31) // 32 for x in xs))


# ---------------------------------------------------------------- scalar ops

def modexp(x: int, e: int, N: int) -> int:
    """x^e mod N by Algorithm 2 (e >= 1, N >= 2)."""
    if e < 1 or N < 2:
        raise ValueError("Algorithm 2 needs e >= 1 and N >= 2")
    n = _nlimbs(N)
    xa, ea, Na = to_limbs(x, _nlimbs(x)), to_limbs(e, _nlimbs(e)), to_limbs(N, n)
    out = np.zeros(n, np.uint32)
    rc = _load().oracle_modexp(_ptr(xa), len(xa), _ptr(ea), len(ea), _ptr(Na), n, _ptr(out))
    if rc:
        raise ValueError(f"oracle_modexp rc={rc}")
    return from_limbs(out)


def mulmod(a: int, b: int, N: int) -> int:
    n = _nlimbs(N, a, b)
    out = np.zeros(n, np.uint32)
    A, B, M = to_limbs(a, n), to_limbs(b, n), to_limbs(N, n)
    if _load().oracle_mulmod(_ptr(A), _ptr(B), _ptr(M), n, _ptr(out)):
        raise ValueError("bad modulus")
    return from_limbs(out)


def divmod_(u: int, v: int) -> tuple[int, int]:
    """(u // v, u % v) by Knuth Algorithm D."""
    nu, nv = _nlimbs(u), _nlimbs(v)
    U, V = to_limbs(u, nu), to_limbs(v, nv)
    nq = max(1, nu - nv + 1)
    q, r = np.zeros(nq, np.uint32), np.zeros(nv, np.uint32)
    if _load().oracle_divmod(_ptr(U), nu, _ptr(V), nv, _ptr(q), nq, _ptr(r), nv):
        raise ZeroDivisionError
    return from_limbs(q), from_limbs(r)


def modinv(a: int, m: int) -> int:
    n = _nlimbs(a, m)
    out = np.zeros(n, np.uint32)
    if _load().oracle_modinv(_ptr(to_limbs(a, n)), _ptr(to_limbs(m, n)), n, _ptr(out)):
        raise ValueError("not invertible")
    return from_limbs(out)


def crt(c: int, dp: int, dq: int, p: int, q: int, qinv: int) -> int:
    """Garner form of the Section 2.1 CRT-RSA decryption."""
    h = _nlimbs(p, q)
    out = np.zeros(2 * h, np.uint32)
    args = [to_limbs(v, h) for v in (dp, dq, p, q, qinv)]
    rc = _load().oracle_crt(_ptr(to_limbs(c, 2 * h)), *[_ptr(a) for a in args], h, _ptr(out))
    if rc:
        raise ValueError(f"oracle_crt rc={rc}")
    return from_limbs(out)


def crt_mp(c: int, primes: list, dexps: list, coefs: list) -> int:
    """Multi-prime CRT decryption of one value (b primes of equal limb count)."""
    b = len(primes)
    h = _nlimbs(*primes)
    cat = lambda vals: np.concatenate([to_limbs(v, h) for v in vals])
    out = np.zeros(b * h, np.uint32)
    R, D, C = cat(primes), cat(dexps), cat(coefs)
    rc = _load().oracle_crt_mp(_ptr(to_limbs(c, b * h)), b, h, _ptr(R), _ptr(D), _ptr(C), _ptr(out))
    if rc:
        raise ValueError(f"oracle_crt_mp rc={rc}")
    return from_limbs(out)


# ---------------------------------------------------------------- keys

class OracleKeys:
    """K key pairs as limb arrays (key-major) and as Python ints.  Multi-prime
    keys (b > 2) hold 'primes', 'dexp' and 'coef' as (K, b * nbits/(32 b))."""

    def __init__(self, K: int, nbits: int, e: int, arrays: dict, b: int = 2):
        self.K, self.nbits, self.e, self.b = K, nbits, e, b
        self.s = nbits // 32
        self.a = arrays  # name -> (K, limbs) uint32

    def prime_list(self, k: int, name: str = "primes") -> list[int]:
        """The b values of `name` (primes, dexp or coef) of key k."""
        h = self.s // self.b
        row = self.a[name][k]
        return [from_limbs(row[i * h:(i + 1) * h]) for i in range(self.b)]

    def ints(self, name: str) -> list[int]:
        return [from_limbs(row) for row in self.a[name]]

    def key(self, k: int) -> dict:
        return {name: from_limbs(self.a[name][k]) for name in self.a} | {"e": self.e}


def keygen(K: int, nbits: int, e: int = 65537, seed: int = 0) -> OracleKeys:
    """Algorithm 1 'Initialization' with the seeded readings of pmk_oracle.c."""
    s, h = nbits // 32, nbits // 64
    arrs = {"N": np.zeros((K, s), np.uint32), "d": np.zeros((K, s), np.uint32)}
    for name in ("p", "q", "dp", "dq", "qinv"):
        arrs[name] = np.zeros((K, h), np.uint32)
    rc = _load().oracle_keygen(K, nbits, e, seed & (2**64 - 1), *[_ptr(arrs[n]) for n in ("N", "d", "p", "q", "dp", "dq", "qinv")])
    if rc:
        raise ValueError(f"oracle_keygen rc={rc}")
    return OracleKeys(K, nbits, e, arrs)


def keygen_mp(K: int, nbits: int, b: int, e: int = 65537, seed: int = 0) -> OracleKeys:
    """Multi-prime key initialisation (Section 2.1): b primes of nbits / b bits per key."""
    s = nbits // 32
    arrs = {n: np.zeros((K, s), np.uint32) for n in ("N", "d", "primes", "dexp", "coef")}
    rc = _load().oracle_keygen_mp(K, nbits, b, e, seed & (2**64 - 1),
                                  *[_ptr(arrs[n]) for n in ("N", "d", "primes", "dexp", "coef")])
    if rc:
        raise ValueError(f"oracle_keygen_mp rc={rc}")
    return OracleKeys(K, nbits, e, arrs, b)


# ---------------------------------------------------------------- split / join

def payload_bytes(nbits: int) -> int:
    """Plaintext bytes per chunk: one byte short of the modulus width, so every chunk is < N."""
    return nbits // 8 - 1


def num_chunks(msg_len: int, nbits: int) -> int:
    P = payload_bytes(nbits)
    return -(-msg_len // P)


def split(msg, nbits: int) -> np.ndarray:
    """Chunk t = bytes [tP, min((t+1)P, L)) read little-endian, zero-extended to nbits/32 limbs."""
    m = np.frombuffer(bytes(msg), dtype=np.uint8) if not isinstance(msg, np.ndarray) else msg.astype(np.uint8, copy=False)
    P, s = payload_bytes(nbits), nbits // 32
    n = num_chunks(len(m), nbits)
    padded = np.zeros(n * P, np.uint8)
    padded[: len(m)] = m
    wide = np.zeros((n, 4 * s), np.uint8)
    wide[:, :P] = padded.reshape(n, P)
    return wide.view("<u4").astype(np.uint32)


def join(chunks: np.ndarray, msg_len: int, nbits: int) -> bytes:
    """Inverse of split: the low P bytes of each chunk, concatenated, cut to msg_len."""
    P, s = payload_bytes(nbits), nbits // 32
    c = np.ascontiguousarray(chunks, dtype="<u4").reshape(-1, s)
    return c.view(np.uint8).reshape(-1, 4 * s)[:, :P].reshape(-1)[:msg_len].tobytes()


# ---------------------------------------------------------------- chunk loops

def _chunk_ranges(n: int, parts: int):
    step = -(-n // max(1, parts))
    return [(a, min(n, a + step)) for a in range(0, n, step)] if n else []


def _run(fn, n: int, threads: int):
    if threads <= 1 or n < 2:
        for a, b in _chunk_ranges(n, 1):
            fn(a, b)
        return
    # ctypes releases the GIL while the C loop runs, so plain threads scale.
    with ThreadPoolExecutor(threads) as ex:
        for f in [ex.submit(fn, a, b) for a, b in _chunk_ranges(n, threads * 4)]:
            f.result()


def modexp_chunks(chunks: np.ndarray, exps: np.ndarray, mods: np.ndarray, threads: int = 1) -> np.ndarray:
    """out_t = chunk_t ^ exps[t mod K] mod mods[t mod K] (Algorithm 1 loops, Algorithm 2 per chunk)."""
    c = np.ascontiguousarray(chunks, dtype=np.uint32)
    n, s = c.shape
    K = mods.shape[0]
    E = np.ascontiguousarray(exps, dtype=np.uint32)
    M = np.ascontiguousarray(mods, dtype=np.uint32)
    assert M.shape == (K, s) and E.shape[0] == K
    out = np.zeros_like(c)
    lib = _load()

    def work(a, b):
        rc = lib.oracle_modexp_chunks(_ptr(c), _ptr(out), s, _ptr(E), E.shape[1], _ptr(M), K, a, b)
        if rc:
            raise ValueError(f"oracle_modexp_chunks rc={rc}")

    _run(work, n, threads)
    return out


def keyed(keys: OracleKeys, key_idx) -> OracleKeys:
    """The key set seen through an explicit chunk-to-key map: row t of every
    key array is key key_idx[t]'s, so the round-robin loops (chunk t -> row
    t mod K, here K = len(key_idx)) bind chunk t to key key_idx[t].  This is
    Algorithm 1 with the i x j reshape of Section 3.1 filled in the caller's
    order instead of column by column."""
    idx = np.asarray(key_idx, dtype=np.int64)
    assert idx.ndim == 1 and (idx >= 0).all() and (idx < keys.K).all()
    return OracleKeys(len(idx), keys.nbits, keys.e, {f: np.ascontiguousarray(v[idx]) for f, v in keys.a.items()},
                      keys.b)


def encrypt_chunks(chunks: np.ndarray, keys: OracleKeys, threads: int = 1, key_idx=None) -> np.ndarray:
    """c_t = m_t^e mod N_k, k = t mod K or key_idx[t]."""
    if key_idx is not None:
        keys = keyed(keys, key_idx)
    e = np.tile(to_limbs(keys.e, 2), (keys.K, 1))
    return modexp_chunks(chunks, e, keys.a["N"], threads)


def decrypt_chunks(chunks: np.ndarray, keys: OracleKeys, use_crt: bool = False, threads: int = 1,
                   key_idx=None) -> np.ndarray:
    """m_t = c_t^d mod N_k (full d, or the Section 2.1 CRT form), k = t mod K or key_idx[t]."""
    if key_idx is not None:
        keys = keyed(keys, key_idx)
    if not use_crt:
        return modexp_chunks(chunks, keys.a["d"], keys.a["N"], threads)
    if "primes" in keys.a:
        return _decrypt_crt_mp(chunks, keys, threads)
    c = np.ascontiguousarray(chunks, dtype=np.uint32)
    n, s = c.shape
    out = np.zeros_like(c)
    lib = _load()
    A = {k: np.ascontiguousarray(keys.a[k]) for k in ("dp", "dq", "p", "q", "qinv")}

    def work(a, b):
        rc = lib.oracle_crt_chunks(_ptr(c), _ptr(out), s, _ptr(A["dp"]), _ptr(A["dq"]), _ptr(A["p"]), _ptr(A["q"]),
                                   _ptr(A["qinv"]), keys.K, a, b)
        if rc:
            raise ValueError(f"oracle_crt_chunks rc={rc}")

    _run(work, n, threads)
    return out


def _decrypt_crt_mp(chunks: np.ndarray, keys: OracleKeys, threads: int) -> np.ndarray:
    c = np.ascontiguousarray(chunks, dtype=np.uint32)
    n, s = c.shape
    out = np.zeros_like(c)
    lib = _load()
    A = {k: np.ascontiguousarray(keys.a[k]) for k in ("primes", "dexp", "coef")}

    def work(a, b):
        rc = lib.oracle_crt_mp_chunks(_ptr(c), _ptr(out), s, keys.b, _ptr(A["primes"]), _ptr(A["dexp"]),
                                      _ptr(A["coef"]), keys.K, a, b)
        if rc:
            raise ValueError(f"oracle_crt_mp_chunks rc={rc}")

    _run(work, n, threads)
    return out


def blind_encrypt_chunks(chunks: np.ndarray, rnd: np.ndarray, keys: OracleKeys, threads: int = 1):
    """Algorithm 1 Encryption with R: returns (C*, C_R), chunk t bound to key t mod K."""
    m = np.ascontiguousarray(chunks, dtype=np.uint32)
    r = np.ascontiguousarray(rnd, dtype=np.uint32)
    n, s = m.shape
    assert r.shape == m.shape
    cstar, cr = np.zeros_like(m), np.zeros_like(m)
    e = np.tile(to_limbs(keys.e, 2), (keys.K, 1))
    M = np.ascontiguousarray(keys.a["N"])
    lib = _load()

    def work(a, b):
        rc = lib.oracle_blind_encrypt_chunks(_ptr(m), _ptr(r), _ptr(cstar), _ptr(cr), s, _ptr(e), 2, _ptr(M), keys.K, a, b)
        if rc:
            raise ValueError(f"oracle_blind_encrypt_chunks rc={rc}")

    _run(work, n, threads)
    return cstar, cr


def blind_decrypt_chunks(cstar: np.ndarray, cr: np.ndarray, keys: OracleKeys, threads: int = 1) -> np.ndarray:
    """Algorithm 1 Decryption with R: r' = c_r^d, m* = c*^d, m' = m* r'^-1 (mod N)."""
    c = np.ascontiguousarray(cstar, dtype=np.uint32)
    q = np.ascontiguousarray(cr, dtype=np.uint32)
    n, s = c.shape
    out = np.zeros_like(c)
    D = np.ascontiguousarray(keys.a["d"])
    M = np.ascontiguousarray(keys.a["N"])
    lib = _load()

    def work(a, b):
        rc = lib.oracle_blind_decrypt_chunks(_ptr(c), _ptr(q), _ptr(out), s, _ptr(D), s, _ptr(M), keys.K, a, b)
        if rc:
            raise ValueError(f"oracle_blind_decrypt_chunks rc={rc}")

    _run(work, n, threads)
    return out
