"""Partitioning one message across ranks (one GPU per rank), with no exchange.

Chunks are independent (Algorithm 1: the loops over chunks parallelise), so a
message shards into contiguous chunk ranges, one per rank.  Chunk t belongs to
key t mod K (Section 3.1), and the kernels bind a call's local chunk j to key
j mod K.  Every range therefore starts at a multiple of K chunks: local j and
global t = start + j then name the same key, and each rank runs split,
encrypt or decrypt and join on its own byte range with the same key set.  The
outputs are disjoint byte ranges of the ciphertext and of the message, so no
collective is needed; a caller that wants the whole result on one device
gathers them.

Host arithmetic only: the work itself runs in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass

from .pmkrsa import num_chunks, payload_bytes


@dataclass(frozen=True)
class Shard:
    rank: int
    chunk_lo: int      # first chunk (a multiple of K)
    chunk_hi: int      # one past the last chunk
    byte_lo: int       # message bytes [byte_lo, byte_hi)
    byte_hi: int

    @property
    def n_chunks(self) -> int:
        return self.chunk_hi - self.chunk_lo

    @property
    def n_bytes(self) -> int:
        return self.byte_hi - self.byte_lo


def shard(msg_len: int, nbits: int, K: int, rank: int, world: int) -> Shard:
    """Rank `rank`'s part of a msg_len-byte message: contiguous chunks in
    blocks of K, the blocks spread as evenly as possible over `world` ranks
    (earlier ranks take one more block when they do not divide evenly).  A
    rank may receive no chunks when the message is short."""
    if world < 1 or not 0 <= rank < world or K < 1 or msg_len < 0:
        raise ValueError("bad shard arguments")
    n = num_chunks(msg_len, nbits)
    P = payload_bytes(nbits)
    blocks = -(-n // K)
    base, extra = divmod(blocks, world)
    b_lo = rank * base + min(rank, extra)
    b_hi = b_lo + base + (1 if rank < extra else 0)
    c_lo, c_hi = min(n, b_lo * K), min(n, b_hi * K)
    return Shard(rank, c_lo, c_hi, min(msg_len, c_lo * P), min(msg_len, c_hi * P))


def shards(msg_len: int, nbits: int, K: int, world: int) -> list[Shard]:
    return [shard(msg_len, nbits, K, r, world) for r in range(world)]
