"""Builds the native PMKRSA library in-tree: ``_build/libpmkrsa.so``.

Every translation unit is compiled with nvcc for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a``), in parallel, then linked
against the shared CUDA runtime (the one torch already loaded).
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libpmkrsa.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cpp", "keygen.cpp", "kernels_aux.cu", "modexp_full.cu", "modexp_crt.cu", "modexp_wide.cu", "peak.cu", "noalloc.cu", "tune.cpp", "batch.cpp",
           "blind.cu", "modexp_latency.cu", "modexp_small.cu", "batch_plan.cpp"]


def _nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _inputs() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    return files + [os.path.join(INCLUDE, "pmkrsa.h"), os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, out: str | None = None,
          defines: tuple = ()) -> str:
    """Compile and link libpmkrsa.so unless it is newer than every source.

    ``out``/``defines`` build a variant elsewhere (for example another row
    form, ``PMK_ROW_FORM=1``) without touching the in-tree library."""
    lib = out or LIB
    if not force and out is None and up_to_date():
        return LIB
    obj_dir = os.path.join(os.path.dirname(lib), "obj" if out is None else "obj_" + os.path.basename(lib))
    os.makedirs(obj_dir, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    common += [f"-D{d}" for d in defines]

    def compile_one(src: str) -> str:
        obj = os.path.join(obj_dir, src + ".o")
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd[1:1] = ["-lineinfo"] + (["-Xptxas", "-v"] if ptxas_info else [])
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
        if verbose and (res.stdout or res.stderr):
            print(res.stdout + res.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    res = subprocess.run([nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs,
                         capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import time

    t0 = time.time()
    print(build(force=True, verbose=True, ptxas_info=True), f"{time.time() - t0:.1f}s")
