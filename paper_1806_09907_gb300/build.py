"""Build libairgb.so in-tree with nvcc for sm_103a (GB300).

Each translation unit under ``csrc/`` is compiled in parallel, then linked
into ``paper_1806_09907_gb300/libairgb.so``. A library is reused only when
the SHA-256 of its sources, headers, compiler flags and nvcc version equals
the one recorded beside it at build time (``<library>.sha256``); a library
copied from elsewhere, or built from other sources, is rebuilt. ``AIRGB_PTXAS_VERBOSE=1`` adds ``-Xptxas -v``
(register / spill / shared-memory report). ``build(checked=True)`` (or
``AIRGB_CHECK=1``) builds the bounds-checked variant ``libairgb_check.so``
(-DAL_CHECK=1: kernels verify their gather indices and record AL_ERR_BOUNDS
instead of reading out of range) beside the regular library.
"""
from __future__ import annotations

import glob
import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libairgb.so")
LIB_CHECK = os.path.join(HERE, "libairgb_check.so")
BUILD_DIR = os.path.join(HERE, "_build")
BUILD_DIR_CHECK = os.path.join(HERE, "_build_check")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libairgb")


def _flags(checked=False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]
    if os.environ.get("AIRGB_PTXAS_VERBOSE") == "1":
        f += ["-Xptxas", "-v"]
    if checked:
        f += ["-DAL_CHECK=1"]
    return f


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _nvcc_version() -> str:
    r = subprocess.run([_nvcc(), "--version"], capture_output=True, text=True)
    return r.stdout


def _digest(checked: bool) -> str:
    """SHA-256 of everything the library is built from."""
    h = hashlib.sha256()
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    deps += glob.glob(os.path.join(INCLUDE, "*.h"))
    for d in sorted(deps):
        h.update(os.path.relpath(d, HERE).encode() + b"\0")
        with open(d, "rb") as f:
            h.update(f.read())
    h.update(" ".join(_flags(checked)).encode())
    h.update(_nvcc_version().encode())
    return h.hexdigest()


def _stamp(lib) -> str:
    return lib + ".sha256"


def _stale(lib=LIB, checked=False) -> bool:
    if not os.path.exists(lib) or not os.path.exists(_stamp(lib)):
        return True
    with open(_stamp(lib)) as f:
        return f.read().strip() != _digest(checked)


def build(force: bool = False, verbose: bool = False, checked: bool = None) -> str:
    """Compile and link libairgb.so (or, checked, libairgb_check.so); returns
    its path."""
    if checked is None:
        checked = os.environ.get("AIRGB_CHECK") == "1"
    lib = LIB_CHECK if checked else LIB
    build_dir = BUILD_DIR_CHECK if checked else BUILD_DIR
    if not force and not _stale(lib, checked):
        return lib
    digest = _digest(checked)
    nvcc = _nvcc()
    os.makedirs(build_dir, exist_ok=True)
    flags = _flags(checked)

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc] + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(_stamp(lib) + ".tmp", "w") as f:
        f.write(digest + "\n")
    os.replace(_stamp(lib) + ".tmp", _stamp(lib))
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
