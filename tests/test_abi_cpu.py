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


@pytest.mark.parametrize("K,nbits,b,e,seed", [(3, 384, 3, 65537, 1), (2, 512, 4, 65537, 2), (2, 768, 3, 3, 3),
                                              (2, 1536, 3, 65537, 4), (1, 2048, 4, 17, 5), (2, 512, 2, 65537, 6),
                                              (1, 3072, 3, 65537, 7)])
def test_library_multiprime_keygen_matches_oracle(P, K, nbits, b, e, seed):
    """Multi-prime key initialisation (Section 2.1): the library's keys equal
    the oracle's limb for limb (primes, N, d, d mod (r_i - 1), the
    recombination coefficients)."""
    lib_keys = P.keygen_host_multiprime(K, nbits, b, e, seed)
    ok = oracle.keygen_mp(K, nbits, b, e, seed)
    for f in ok.a:
        assert np.array_equal(lib_keys[f], ok.a[f]), f


def test_multiprime_two_primes_equal_keygen(P):
    mp = P.keygen_host_multiprime(3, 1024, 2, 65537, 9)
    two = P.keygen_host(3, 1024, 65537, 9)
    h = 16
    assert np.array_equal(mp["N"], two["N"]) and np.array_equal(mp["d"], two["d"])
    assert np.array_equal(mp["primes"][:, :h], two["p"]) and np.array_equal(mp["primes"][:, h:], two["q"])
    assert np.array_equal(mp["coef"][:, :h], two["qinv"])


def test_multiprime_keygen_argument_errors(P):
    for bad in [(1, 2048, 3), (1, 768, 5), (1, 768, 1), (1, 640, 4), (0, 768, 3), (16384, 768, 3), (1, 9216, 3)]:
        with pytest.raises(P.PMKError):
            P.keygen_host_multiprime(*bad, e=65537, seed=1)
    with pytest.raises(P.PMKError):
        P.keygen_host_multiprime(1, 768, 3, e=4, seed=1)


def test_no_context_without_gpu(P):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(P.PMKError):
        P.Context(0)  # no silent CPU path


def test_tune_cache_keys_and_persistence(P, tmp_path):
    """The autotuner cache keys results by GPU, width, prime count, mode and
    power-of-two batch bucket, and survives a reload from disk."""
    path = str(tmp_path / "tune.json")
    c = P.TuneCache(path)
    k1 = c.key("GB300", 2048, 2, "crt", 4113)
    assert k1 == c.key("GB300", 2048, 2, "crt", 8192) != c.key("GB300", 2048, 2, "crt", 8193)
    assert k1 != c.key("GB300", 2048, 3, "crt", 4113) != c.key("B200", 2048, 2, "crt", 4113)
    assert c.key("GB300", 2048, 2, "decrypt", 1) == "GB300|2048|2|decrypt|1"
    assert c.get(k1) is None
    c.put(k1, {"tpi": 4, "form": 1, "window": 4, "ms": 4.8})
    k2 = c.key("GB300", 4096, 2, "decrypt", 100)
    c.put(k2, {"tpi": 16, "form": 0, "ms": 9.5})  # no window given: the default bound, 5
    again = P.TuneCache(path)
    assert again.get(k1) == {"tpi": 4, "form": 1, "window": 4, "ms": 4.8}
    assert again.get(k2) == {"tpi": 16, "form": 0, "window": 5, "ms": 9.5}
    (tmp_path / "bad.json").write_text("not json")
    assert P.TuneCache(str(tmp_path / "bad.json")).entries == {}


def test_header_is_plain_c_and_links_from_c(P, tmp_path):
    """A C99 program includes include/pmkrsa.h (no C++), links libpmkrsa.so
    and runs the host-only entry points; its key equals the oracle's."""
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2111_11924_gb300 import _native_build as NB

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lib = NB.LIB
    exe = str(tmp_path / "abi_host_calls")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-o", exe,
                           os.path.join(root, "tests", "c", "abi_host_calls.c"), "-I", os.path.join(root, "include"),
                           lib, "-Wl,-rpath," + os.path.dirname(lib)])
    out = subprocess.run([exe, "0x1234"], capture_output=True, text=True, check=True).stdout.split("\n")
    assert out[0] == "payload 255 chunks 4113"
    assert "modulus" in out[1] and out[2] == "keygen 0" and out[4] == f"bad_width {P.pmkrsa.PMK_EINVAL}"
    limbs = [int(x, 16) for x in out[3].split()[1:]]
    ok = oracle.keygen(2, 512, 65537, 0x1234)
    assert limbs == [int(v) for v in ok.a["N"][0]]


def test_geometry_calls_host_only(P):
    """The geometry and window-bound calls reject a NULL context and bad
    arguments on the host; the compiled geometry list needs no GPU."""
    import ctypes

    import paper_2111_11924_gb300.pmkrsa as B

    lib = P.load_library()
    w = (ctypes.c_uint32 * 1)()
    assert lib.pmk_set_kernel_window(None, 32, 1, 4) == B.PMK_EINVAL
    assert lib.pmk_get_kernel_window(None, 32, 1, w) == B.PMK_EINVAL
    assert lib.pmk_set_kernel_config(None, 64, 0, 8, 1) == B.PMK_EINVAL
    assert lib.pmk_list_kernel_configs(64, 0, None, None, -1) == B.PMK_EINVAL
    full64 = P.kernel_configs(64, False)
    assert (8, 1) in full64 and len(full64) == len(set(full64))  # one entry per geometry, whatever the tables
    crt32 = P.kernel_configs(32, True)
    assert (4, 1) in crt32 and len(crt32) == len(set(crt32))  # small-table twins are not listed twice
    assert P.kernel_configs(40, True) == []


def test_exponent_schedules_replay_to_their_exponents(tmp_path):
    """The host's window schedules (tests/c/schedule_check.cpp, built against
    keygen.cpp with g++): replayed on plain integers, every single-exponent
    schedule (window bounds 1-5) and every joint schedule of the blinded CRT
    decryption gives back its exponents, with each odd-power index inside
    the table bound, over 1-256-limb exponents (random, sparse, dense and
    special values)."""
    import shutil
    import subprocess

    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    from paper_2111_11924_gb300 import _native_build as NB

    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    exe = str(tmp_path / "schedule_check")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-Wall", "-Wextra", "-Werror", "-o", exe,
                           os.path.join(ROOT, "tests", "c", "schedule_check.cpp"),
                           os.path.join(NB.CSRC, "keygen.cpp"), "-I", os.path.join(ROOT, "include"), "-I", NB.CSRC,
                           "-I", cuda_inc, "-lpthread"])
    res = subprocess.run([exe], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout
    assert res.stdout.strip().endswith("0 failures") and int(res.stdout.split()[0]) >= 1000


def test_unexported_key_constants_from_their_definitions(tmp_path):
    """The per-key constants the kernels use but the C ABI does not export
    (Montgomery constants, R^2 / R_h^2 / R_h^3, the CRT recombination rows,
    d mod (r_i - 1), the Garner coefficients), recomputed from their
    definitions with 128-bit integers on keys whose primes fit in 64 bits
    (tests/c/keyconst_check.cpp, built against keygen.cpp with g++)."""
    import shutil
    import subprocess

    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    from paper_2111_11924_gb300 import _native_build as NB

    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    exe = str(tmp_path / "keyconst_check")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-Wall", "-Wextra", "-Werror", "-o", exe,
                           os.path.join(ROOT, "tests", "c", "keyconst_check.cpp"),
                           os.path.join(NB.CSRC, "keygen.cpp"), "-I", os.path.join(ROOT, "include"), "-I", NB.CSRC,
                           "-I", cuda_inc, "-lpthread"])
    res = subprocess.run([exe], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout
    assert res.stdout.strip().endswith("0 failures") and int(res.stdout.split()[0]) >= 500


def test_batch_planner_covers_every_chunk_once(tmp_path):
    """The batch planner (batch_plan.cpp, built with g++ against
    tests/c/batch_plan_check.cpp and stand-in geometry / capacity functions)
    over 300 random job mixes: grid launches exactly for jobs of several
    GPU-fulls, every other chunk and prime in exactly one task of its key,
    task sizes within a warp, groups widest first with decryptions first,
    and refusal of widths without a geometry or capacity."""
    import shutil
    import subprocess

    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    from paper_2111_11924_gb300 import _native_build as NB

    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    exe = str(tmp_path / "batch_plan_check")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-Wall", "-Wextra", "-Werror", "-o", exe,
                           os.path.join(ROOT, "tests", "c", "batch_plan_check.cpp"),
                           os.path.join(NB.CSRC, "batch_plan.cpp"), "-I", os.path.join(ROOT, "include"), "-I",
                           NB.CSRC, "-I", cuda_inc])
    res = subprocess.run([exe], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout
    assert res.stdout.strip().endswith("0 failures") and int(res.stdout.split()[0]) >= 1_000_000


def test_host_buffer_checks_reject_mismatched_buffers():
    """The binding checks host buffers before a *_host call would read past
    them: shape and dtype of the limb buffer, dtype and chunk count of the
    message, contiguity and device."""
    import torch

    from paper_2111_11924_gb300 import pmkrsa

    good = torch.zeros((5, 32), dtype=torch.int32)
    assert pmkrsa.host_limb_buffer(good, 1024) == 5
    for bad in (torch.zeros((5, 64), dtype=torch.int32),      # another key width
                torch.zeros((5, 32), dtype=torch.int64),      # wrong dtype
                torch.zeros((32, 5), dtype=torch.int32).t(),  # not contiguous
                torch.zeros(160, dtype=torch.int32)):         # not 2-D
        with pytest.raises(ValueError):
            pmkrsa.host_limb_buffer(bad, 1024)
    assert pmkrsa.chunk_shape(good, 1024, 5) == 5
    for bad, n in ((good, 4), (torch.zeros((5, 64), dtype=torch.int32), 5), (torch.zeros(160), None), ([0], None)):
        with pytest.raises(ValueError):
            pmkrsa.chunk_shape(bad, 1024, n)
    msg = torch.zeros(5 * 127 - 3, dtype=torch.uint8)
    assert pmkrsa.host_message_buffer(msg, 5, 1024) == 5 * 127 - 3
    for bad, n in ((torch.zeros(5 * 127 + 1, dtype=torch.uint8), 5),  # one chunk too many
                   (torch.zeros(600, dtype=torch.int8), 5),           # wrong dtype
                   (torch.zeros((2, 300), dtype=torch.uint8)[:, :200], 4)):  # not contiguous
        with pytest.raises(ValueError):
            pmkrsa.host_message_buffer(bad, n, 1024)


def test_blob_round_trip_from_c(P, tmp_path):
    """A C99 program writes a key-set blob with its own writer, imports it
    host-only, exports it and gets the same bytes; a corrupted or
    inconsistent blob is refused."""
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2111_11924_gb300 import _native_build as NB

    exe = str(tmp_path / "blob_roundtrip")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-o", exe,
                           os.path.join(ROOT, "tests", "c", "blob_roundtrip.c"), "-I", os.path.join(ROOT, "include"),
                           NB.LIB, "-Wl,-rpath," + os.path.dirname(NB.LIB)])
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    einval = P.pmkrsa.PMK_EINVAL
    assert out[0] == "keygen 0" and out[1] == "import 0"
    assert out[2] == f"export 0 0 size {32 + 20 * 3 * 24 + 8} same"
    assert out[3] == f"corrupt {einval}" and out[4] == f"inconsistent {einval}"


def _fnv1a64(b: bytes) -> int:
    h = 0xCBF29CE484222325
    for x in b:
        h = ((h ^ x) * 0x100000001B3) & (2**64 - 1)
    return h


def _oracle_blob(ok, b: int) -> bytes:
    """The documented blob layout written from the oracle's key material."""
    import struct

    s = ok.nbits // 32
    rows = []
    for k in range(ok.K):
        if b == 2:
            primes = np.concatenate([ok.a["p"][k], ok.a["q"][k]])
            dexp = np.concatenate([ok.a["dp"][k], ok.a["dq"][k]])
            coef = np.concatenate([ok.a["qinv"][k], np.zeros(s // 2, np.uint32)])
        else:
            primes, dexp, coef = ok.a["primes"][k], ok.a["dexp"][k], ok.a["coef"][k]
        rows += [ok.a["N"][k], ok.a["d"][k], primes, dexp, coef]
    body = b"PMKK" + struct.pack("<5IQ", 1, ok.K, ok.nbits, b, 0, ok.e) + \
        b"".join(np.asarray(r, dtype="<u4").tobytes() for r in rows)
    return body + struct.pack("<Q", _fnv1a64(body))


@pytest.mark.parametrize("K,nbits,b,seed", [(3, 512, 2, 11), (2, 768, 3, 12), (2, 1024, 4, 13)])
def test_blob_matches_oracle_key_material(P, K, nbits, b, seed):
    """A blob written from the oracle's keys imports into a key set whose
    exported material is the oracle's, and exports back to the same bytes."""
    ok = oracle.keygen(K, nbits, 65537, seed) if b == 2 else oracle.keygen_mp(K, nbits, b, 65537, seed)
    blob = _oracle_blob(ok, b)
    ks = P.import_keyset_host(blob)
    assert (ks.K, ks.nbits, ks.nprimes, ks.e) == (K, nbits, b, 65537)
    assert ks.export_blob() == blob
    ex = ks.export()
    for f in ok.a:
        assert np.array_equal(ex[f], ok.a[f]), f
    ks.free()


def test_blob_rejections(P):
    ok = oracle.keygen(2, 512, 65537, 21)
    blob = bytearray(_oracle_blob(ok, 2))
    for mutate in (lambda x: x.__setitem__(0, ord("Q")),              # magic
                   lambda x: x.__setitem__(4, 2),                     # version
                   lambda x: x.__setitem__(len(x) - 1, x[-1] ^ 1),    # hash
                   lambda x: x.__setitem__(slice(len(x) - 9, len(x) - 8), b"")):  # length
        bad = bytearray(blob)
        mutate(bad)
        with pytest.raises(P.PMKError) as err:
            P.import_keyset_host(bytes(bad))
        assert err.value.code == P.pmkrsa.PMK_EINVAL


def test_host_only_key_set_is_refused_by_device_calls(P):
    """A key set imported without a context has no device tables: the
    allocation-free decryption refuses it (EINVAL) before any device work,
    so the refusal is visible on a machine with no GPU."""
    import torch

    ok = oracle.keygen(2, 512, 65537, 22)
    ks = P.import_keyset_host(_oracle_blob(ok, 2))
    n = 3
    cipher = torch.zeros((n, 512 // 32), dtype=torch.int32)
    msg = torch.zeros(n * (512 // 8 - 1), dtype=torch.uint8)
    for crt in (False, True):
        assert P.pmkrsa.decrypt_message_host_noalloc(ks, cipher, msg, use_crt=crt) == P.pmkrsa.PMK_EINVAL
    empty = torch.zeros((0, 512 // 32), dtype=torch.int32)
    assert P.pmkrsa.decrypt_message_host_noalloc(ks, empty, torch.zeros(0, dtype=torch.uint8)) == P.pmkrsa.PMK_EINVAL
    ks.free()
