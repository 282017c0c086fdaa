"""Sharding one message across ranks: the shards partition the chunks, start
on multiples of K, and the per-shard results (computed here by the oracle,
rank by rank) concatenate to the whole message's results."""
import numpy as np
import pytest

import oracle
from paper_2111_11924_gb300 import sharding as SH


@pytest.mark.parametrize("L,nbits,K,world", [(0, 1024, 4, 2), (1, 1024, 4, 3), (32768, 1024, 4, 2),
                                             (32768, 1024, 4, 7), (1 << 20, 2048, 8, 4), (100000, 2048, 16, 8),
                                             (5000, 512, 3, 5)])
def test_shards_partition_on_key_block_boundaries(L, nbits, K, world):
    n = oracle.num_chunks(L, nbits)
    P = oracle.payload_bytes(nbits)
    parts = SH.shards(L, nbits, K, world)
    assert parts[0].chunk_lo == 0 and parts[-1].chunk_hi == n
    for a, b in zip(parts, parts[1:]):
        assert a.chunk_hi == b.chunk_lo and a.byte_hi == b.byte_lo
    for p in parts:
        assert p.chunk_lo % K == 0 or p.chunk_lo == n
        assert p.byte_lo == min(L, p.chunk_lo * P) and p.byte_hi == min(L, p.chunk_hi * P)
        assert p.n_chunks == oracle.num_chunks(p.n_bytes, nbits)  # a shard is a message of its own
    sizes = [p.n_chunks for p in parts]
    assert max(sizes) - min(sizes) <= 2 * K - 1  # one block of K, plus a partial last block


def test_sharded_encryption_equals_whole_message():
    """Each rank encrypts its byte range with the same keys (oracle on the
    CPU); the ciphertext chunks concatenate to the whole message's, because
    every shard starts on a multiple of K."""
    nbits, K, L, world = 512, 3, 7000, 4
    keys = oracle.keygen(K, nbits, 65537, 77)
    msg = np.random.default_rng(3).integers(0, 256, L, dtype=np.uint8)
    whole = oracle.encrypt_chunks(oracle.split(msg, nbits), keys)
    parts = []
    for p in SH.shards(L, nbits, K, world):
        part = msg[p.byte_lo:p.byte_hi]
        if len(part):
            parts.append(oracle.encrypt_chunks(oracle.split(part, nbits), keys))
    assert np.array_equal(np.concatenate(parts), whole)
    back = b"".join(oracle.join(oracle.decrypt_chunks(c, keys), len(c) * oracle.payload_bytes(nbits), nbits)
                    for c in parts)
    assert back[:L] == msg.tobytes()


def test_bad_arguments():
    for args in [(10, 1024, 0, 0, 1), (10, 1024, 4, 2, 2), (10, 1024, 4, 0, 0), (-1, 1024, 4, 0, 1)]:
        with pytest.raises(ValueError):
            SH.shard(*args)
