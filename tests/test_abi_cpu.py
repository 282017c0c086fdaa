"""CPU-side checks of the native library: it loads, exports every symbol the
header declares, and its host-only logic (chunk arithmetic, key
initialisation) agrees with the oracle.  No call here touches a GPU."""
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2111_11924_gb300 import _native_build

    _native_build.build()  # no-op when up to date; nvcc cross-compiles without a GPU
    import paper_2111_11924_gb300 as P

    return P


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pmkrsa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pmk_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(P):
    lib = P.load_library()
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(P):
    import paper_2111_11924_gb300.pmkrsa as B

    src = open(B.__file__).read()
    assert all(f'"{n}"' in src for n in declared_functions())


@pytest.mark.parametrize("L,nbits", [(0, 1024), (1, 1024), (32768, 1024), (1048576, 2048), (104857600, 2048),
                                     (255, 2048), (256, 2048), (1000, 128)])
def test_chunk_arithmetic_matches_oracle(P, L, nbits):
    assert P.num_chunks(L, nbits) == oracle.num_chunks(L, nbits)
    assert P.payload_bytes(nbits) == oracle.payload_bytes(nbits)


def test_strerror(P):
    assert P.strerror(0) == "ok"
    assert "modulus" in P.strerror(-2)
    assert P.strerror(12345) == "unknown error"


@pytest.mark.parametrize("K,nbits,e,seed", [(3, 128, 65537, 1), (4, 256, 65537, 2), (2, 512, 3, 3),
                                            (2, 1024, 65537, 0x50444D4B00000101), (1, 2048, 65537, 5),
                                            (2, 384, 17, 6)])
def test_library_keygen_matches_oracle(P, K, nbits, e, seed):
    """Same seeded key initialisation, two independent implementations
    (library: Montgomery arithmetic and d = (k phi + 1)/e; oracle: Knuth
    division and extended Euclid), identical keys."""
    lib_keys = P.keygen_host(K, nbits, e, seed)
    ok = oracle.keygen(K, nbits, e, seed)
    for f in ok.a:
        assert np.array_equal(lib_keys[f], ok.a[f]), f


def test_keygen_argument_errors(P):
    for bad in [(0, 1024, 65537), (1, 1000, 65537), (1, 1024, 4), (1, 1024, 1), (1, 16384, 65537), (1, 1024, 1 << 33)]:
        with pytest.raises(P.PMKError):
            P.keygen_host(*bad, seed=1)


def test_no_context_without_gpu(P):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(P.PMKError):
        P.Context(0)  # no silent CPU path
