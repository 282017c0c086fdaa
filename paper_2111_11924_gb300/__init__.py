"""GB300-native PMKRSA hot path ("A Variant RSA Acceleration with Parallelization", arXiv 2111.11924).

A message is split into chunks, chunk t is bound to key pair t mod K (or to
a key the caller names per chunk), and every chunk is one modular
exponentiation (Section 3.1, Algorithm 1).  All of that runs in the
hand-written sm_103a kernels of ``libpmkrsa.so``; this
module is argument marshalling over its C ABI (``include/pmkrsa.h``) with
torch tensors as device buffers and torch streams as CUDA streams.  There is
no CPU fallback: if the native library is missing, importing this package
fails.
"""
from __future__ import annotations

from .pmkrsa import (  # noqa: F401
    PMKError,
    Context,
    KeySet,
    keygen_host,
    keygen_host_multiprime,
    import_keyset_host,
    TuneCache,
    kernel_configs,
    load_library,
    num_chunks,
    payload_bytes,
    strerror,
)
from . import sharding  # noqa: F401

__all__ = ["PMKError", "Context", "KeySet", "keygen_host", "keygen_host_multiprime", "import_keyset_host", "TuneCache", "kernel_configs", "load_library", "num_chunks", "payload_bytes", "strerror", "sharding"]
