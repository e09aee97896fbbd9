"""In-tree build of libsbio.so for sm_103a (nvcc only, no cmake).

Each CUDA translation unit is compiled in parallel to an object file under
``paper_2506_20809_gb300/_build`` and linked into
``paper_2506_20809_gb300/libsbio.so``.  Run ``python -m
paper_2506_20809_gb300.build`` or call :func:`build`.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsbio.so")
LIB_HASH = LIB + ".srchash"
SOURCES = ["sbio_geom.cu", "sbio_laplace.cu", "sbio_stokes.cu", "sbio_noalloc.cu", "sbio_batch.cu", "sbio_server.cu",
           "sbio_deriv.cu", "sbio_targets.cu", "sbio_solve.cu", "sbio_stokes_points.cu", "sbio_stokes_dl.cu",
           "sbio_peaks.cu", "sbio_tree.cu"]
# near-field kernels, split by expansion order so that the unrolled variants compile in parallel
SOURCES += [f"sbio_near_p{c}.cu" for c in "abcd"]
SOURCES += [f"sbio_deriv_near_p{c}.cu" for c in "ab"]
SOURCES += [f"sbio_stokes_near_p{c}.cu" for c in "abc"]
SOURCES += [f"sbio_stokes_points_p{c}.cu" for c in "abc"]
SOURCES += [f"sbio_stokes_dl_near_p{c}.cu" for c in "abcdefghij"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags() -> list[str]:
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", os.path.join(ROOT, "include")]


def _object_key(src: str, common: str) -> str:
    """Hash of one translation unit: its source plus every header of the
    package and the flags (`common`), so an object is rebuilt whenever
    anything it may include changes."""
    h = hashlib.sha256(common.encode())
    with open(os.path.join(CSRC, src), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()


def _headers_and_flags() -> str:
    h = hashlib.sha256()
    for f in sorted(f for f in os.listdir(CSRC) if f.endswith(".cuh")):
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    with open(os.path.join(ROOT, "include", "sbio.h"), "rb") as fh:
        h.update(fh.read())
    # objects built on another host architecture are never reused
    h.update(" ".join(_flags()).encode() + nvcc_path().encode() + platform.machine().encode())
    return h.hexdigest()


def _compile(src: str, verbose_ptxas: bool, common: str = "") -> tuple[str, str]:
    obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
    key = _object_key(src, common)
    if not verbose_ptxas and os.path.exists(obj) and os.path.exists(obj + ".hash"):
        with open(obj + ".hash") as fh:
            if fh.read().strip() == key:
                return obj, ""
    cmd = [nvcc_path(), *_flags(), "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    with open(obj + ".hash", "w") as fh:
        fh.write(key + "\n")
    return obj, r.stderr


def source_hash() -> str:
    """SHA-256 over every source and header the library is built from, the
    list of translation units and the nvcc command line (compiler path and
    version included), so that a library built from other sources or flags is
    never reused."""
    h = hashlib.sha256()
    files = sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh")))
    for f in files:
        h.update(f.encode() + b"\0")
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(ROOT, "include", "sbio.h"), "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(SOURCES).encode())
    h.update(" ".join(_flags()).encode())
    nv = nvcc_path()
    ver = subprocess.run([nv, "--version"], capture_output=True, text=True).stdout
    h.update(nv.encode() + ver.encode() + platform.machine().encode())
    return h.hexdigest()


def build(verbose_ptxas: bool = False, force: bool = False) -> str:
    """Compile every translation unit and link libsbio.so; returns its path.
    An existing library is reused only if the hash stored beside it matches
    the current sources and flags (never by file times)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    want = source_hash()
    if not force and os.path.exists(LIB) and os.path.exists(LIB_HASH):
        with open(LIB_HASH) as fh:
            if fh.read().strip() == want:
                return LIB
    common = _headers_and_flags()
    # objects are reused only when their own key matches (never by file times)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose_ptxas, common), SOURCES))
    objs = [o for o, _ in results]
    if verbose_ptxas:
        for _, log in results:
            sys.stderr.write(log)
    tmp = LIB + ".tmp"
    r = subprocess.run([nvcc_path(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(LIB_HASH + ".tmp", "w") as fh:
        fh.write(want + "\n")
    os.replace(LIB_HASH + ".tmp", LIB_HASH)
    return LIB


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv, force=True))
