"""Build the sm_103a CUDA libraries in-tree.

    python -m paper_2512_09664_b300.build [--force] [--ptxas-v]

* ``paper_2512_09664_b300/libsynthpix.so``: the renderer (``csrc/*.cu``),
  the C ABI of ``include/synthpix.h``.
* ``paper_2512_09664_b300/libsynthpix_probe.so``: the ALU throughput probes
  of ``measure/`` (measurement support for the benchmark only).
* ``paper_2512_09664_b300/libsynthpix_smallbins.so``: the renderer with fixed
  bins too small for their records (``SPX_SMALL_FIXED_BINS``), so that the
  tests can run the exact rebinning after an overflow, which the product
  library's bin capacities make all but impossible to reach.  Only the units
  that size the bins are compiled again.

nvcc cross-compiles for sm_103a without a GPU.  Each translation unit is
compiled to an object of its own (in parallel, into ``_build/``; a unit is
rebuilt when it or any header changed), then linked.  The libraries link
the shared CUDA runtime (libcudart.so.13), the same one PyTorch loads.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
MEASURE = os.path.join(PKG, "measure")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libsynthpix.so")
PROBE_LIB = os.path.join(PKG, "libsynthpix_probe.so")
SMALLBINS_LIB = os.path.join(PKG, "libsynthpix_smallbins.so")
SMALLBINS_UNITS = ("prep.cu", "api.cu")  # the units that size the fixed bins
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMPILE_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                 "--expt-relaxed-constexpr"]
LINK_FLAGS = ["-shared", "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def probe_sources():
    return sorted(glob.glob(os.path.join(MEASURE, "*.cu")))


def _headers(folder):
    return glob.glob(os.path.join(folder, "*.cuh")) + glob.glob(os.path.join(folder, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _newer(paths, t):
    return any(os.path.getmtime(p) > t for p in paths)


def _stale() -> bool:
    for lib, srcs, folder in ((LIB, sources(), CSRC), (PROBE_LIB, probe_sources(), MEASURE),
                              (SMALLBINS_LIB, sources(), CSRC)):
        if not os.path.exists(lib) or _newer(srcs + _headers(folder), os.path.getmtime(lib)):
            return True
    return False


def _obj(src, tag):
    return os.path.join(BUILD, f"{tag}_{os.path.splitext(os.path.basename(src))[0]}.o")


def _compile(src, obj, inc, extra, verbose):
    cmd = [NVCC, *ARCH_FLAGS, *COMPILE_FLAGS, "-I" + INCLUDE, "-I" + inc, *extra, "-c", src, "-o", obj + ".tmp"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(obj + ".tmp", obj)
    return obj


def _build_lib(lib, srcs, folder, tag, force, verbose, extra, variant=None):
    """variant: None, or (tag, units, flags): those units compiled again with the flags
    (objects tagged `tag`), the others shared with the main build."""
    os.makedirs(BUILD, exist_ok=True)
    hdr_t = max([os.path.getmtime(h) for h in _headers(folder)] or [0.0])

    def obj_of(s):
        if variant and os.path.basename(s) in variant[1]:
            return _obj(s, variant[0])
        return _obj(s, tag)

    jobs = []
    for s in srcs:
        o = obj_of(s)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr_t):
            flags = list(extra) + (list(variant[2]) if variant and o != _obj(s, tag) else [])
            jobs.append((s, o, flags))
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for f in [ex.submit(_compile, s, o, folder, fl, verbose) for s, o, fl in jobs]:
            f.result()
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH_FLAGS, *LINK_FLAGS, *[obj_of(s) for s in srcs], "-o", tmp]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and not _stale():
        return LIB
    _build_lib(LIB, sources(), CSRC, "spx", force, verbose, list(extra))
    _build_lib(PROBE_LIB, probe_sources(), MEASURE, "probe", force, verbose, list(extra))
    _build_lib(SMALLBINS_LIB, sources(), CSRC, "spx", force, verbose, list(extra),
               variant=("smallbins", SMALLBINS_UNITS, ["-DSPX_SMALL_FIXED_BINS"]))
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else [])
    print(LIB)
    print(PROBE_LIB)
    print(SMALLBINS_LIB)
