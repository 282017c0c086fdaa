"""Seeded synthetic workloads (inputs only -- none of the method's arithmetic).

The paper's experiments encrypt randomly generated files (Section 4: 100 KB
plaintexts for Tables 1-2, 1-100 MB files for Table 3), so uniform random
bytes stand in for them.  Each workload names its sizes; message bytes come
from numpy's PCG64 seeded with ``MSG_SEED_BASE + id`` and keys from the
library / oracle keygen seeded with ``KEY_SEED_BASE + id`` (both sides
implement the same seeded key initialisation).  Both the CUDA path and the
oracle read their inputs from here.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

MSG_SEED_BASE = 0x50444D4B00000000
KEY_SEED_BASE = 0x50444D4B00000100


@dataclass(frozen=True)
class Workload:
    id: int
    name: str
    msg_bytes: int
    K: int
    nbits: int
    e: int = 65537

    @property
    def payload(self) -> int:
        return self.nbits // 8 - 1

    @property
    def n_chunks(self) -> int:
        return -(-self.msg_bytes // self.payload)

    @property
    def limbs(self) -> int:
        return self.nbits // 32

    @property
    def msg_seed(self) -> int:
        return MSG_SEED_BASE + self.id

    @property
    def key_seed(self) -> int:
        return KEY_SEED_BASE + self.id

    def message(self) -> np.ndarray:
        return np.random.default_rng(self.msg_seed).integers(0, 256, self.msg_bytes, dtype=np.uint8)

    def describe(self) -> dict:
        return {"workload": self.name, "msg_bytes": self.msg_bytes, "chunks": self.n_chunks, "keys": self.K,
                "key_bits": self.nbits, "e": self.e, "chunk_payload_bytes": self.payload,
                "key_assignment": "round-robin t mod K", "msg_seed": hex(self.msg_seed), "key_seed": hex(self.key_seed)}


# 32 KiB, K = 4, 1024-bit keys: small enough for a full oracle comparison.
SMALL_1024 = Workload(1, "pmkrsa-32KiB-K4-1024bit", 32 * 1024, 4, 1024)
# 1 MiB, K = 8, 2048-bit keys: the headline decrypt workload.
FILE_1MIB_2048 = Workload(2, "pmkrsa-1MiB-K8-2048bit", 1 << 20, 8, 2048)
# 100 MiB, K = 16, 2048-bit keys: the largest file of Table 3.
FILE_100MIB_2048 = Workload(3, "pmkrsa-100MiB-K16-2048bit", 100 << 20, 16, 2048)

ALL = {w.name: w for w in (SMALL_1024, FILE_1MIB_2048, FILE_100MIB_2048)}


def random_below(rng: np.random.Generator, bound: int) -> int:
    """Uniform integer in [0, bound) from the generator (rejection on whole bytes)."""
    nbytes = (bound.bit_length() + 7) // 8
    while True:
        v = int.from_bytes(rng.bytes(nbytes), "little") & ((1 << bound.bit_length()) - 1)
        if v < bound:
            return v


def blinding_values(n_chunks: int, nbits: int, seed: int) -> np.ndarray:
    """The random matrix R of Algorithm 1 as an input: one value per chunk,
    uniform below 2^(nbits - 8) (so below every nbits-bit modulus), as
    (n_chunks, nbits/32) little-endian uint32 limbs."""
    s = nbits // 32
    nbytes = nbits // 8 - 1
    raw = np.zeros((n_chunks, 4 * s), np.uint8)
    raw[:, :nbytes] = np.random.default_rng(seed).integers(0, 256, (n_chunks, nbytes), dtype=np.uint8)
    return raw.view("<u4").astype(np.uint32)
