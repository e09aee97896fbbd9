"""In-tree build of libsbio.so for sm_103a (nvcc only, no cmake).

Each CUDA translation unit is compiled in parallel to an object file under
``paper_2506_20809_gb300/_build`` and linked into
``paper_2506_20809_gb300/libsbio.so``.  Run ``python -m
paper_2506_20809_gb300.build`` or call :func:`build`.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsbio.so")
SOURCES = ["sbio_geom.cu", "sbio_laplace.cu", "sbio_stokes.cu", "sbio_noalloc.cu", "sbio_batch.cu", "sbio_server.cu",
           "sbio_deriv.cu", "sbio_targets.cu", "sbio_solve.cu", "sbio_stokes_points.cu", "sbio_stokes_dl.cu"]
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


def _compile(src: str, verbose_ptxas: bool) -> tuple[str, str]:
    obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc_path(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
           "-I", os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj, r.stderr


def build(verbose_ptxas: bool = False, force: bool = False) -> str:
    """Compile every translation unit and link libsbio.so; returns its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    deps.append(os.path.join(ROOT, "include", "sbio.h"))
    if not force and os.path.exists(LIB):
        t_lib = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) < t_lib for d in deps):
            return LIB
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose_ptxas), SOURCES))
    objs = [o for o, _ in results]
    if verbose_ptxas:
        for _, log in results:
            sys.stderr.write(log)
    tmp = LIB + ".tmp"
    r = subprocess.run([nvcc_path(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv, force=True))
