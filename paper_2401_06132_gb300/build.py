"""Builds the in-tree CUDA library libfrgb300.so for sm_103a (nvcc; translation units in parallel)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfrgb300.so")
# variants: "" the release library; "bounds" the bounds-checking build (FR_DEBUG_BOUNDS: element
# offsets and partner indices checked on the device, failures reported as FR_EBOUNDS)
VARIANTS = {"": ([], BUILD, LIB), "bounds": (["-DFR_DEBUG_BOUNDS"], os.path.join(BUILD, "bounds"),
                                             os.path.join(HERE, "libfrgb300_bounds.so"))}
SOURCES = ["fr_api.cu", "fr_hex.cu", "fr_pri.cu", "fr_dense.cu", "fr_probe.cu", "fr_basis.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"] + ARCH


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _headers() -> list:
    """Every header a translation unit can include: the library's own and the public ABI header."""
    inc = os.path.join(HERE, "..", "include")
    return sorted(os.path.join(d, f) for d in (CSRC, inc) for f in os.listdir(d) if f.endswith((".h", ".cuh")))


def _compile(src: str, extra, bdir: str = BUILD) -> str:
    obj = os.path.join(bdir, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    cmd = [nvcc()] + NVCC_FLAGS + list(extra) + ["-c", path, "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc(), "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-x", "c++", "-c", path, "-o", obj]
    # an object is reused only if it is newer than its source and every header, and was compiled
    # with the same command line
    stamp = obj + ".cmd"
    deps = [path] + _headers()
    if (os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == " ".join(cmd)
            and all(os.path.getmtime(obj) >= os.path.getmtime(d) for d in deps)):
        return obj
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    with open(stamp, "w") as f:
        f.write(" ".join(cmd))
    return obj


def build(verbose: bool = False, extra=(), variant: str = "") -> str:
    flags, bdir, lib = VARIANTS[variant]
    os.makedirs(bdir, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, list(flags) + list(extra), bdir), SOURCES))
    if not os.path.exists(lib) or any(os.path.getmtime(o) > os.path.getmtime(lib) for o in objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", lib + ".tmp"] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(lib + ".tmp", lib)
    if verbose:
        print("built", lib)
    return lib


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
