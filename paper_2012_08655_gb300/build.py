"""In-tree build of libfovea.so (hand-written sm_103a CUDA + C++ host code).

Every translation unit is compiled in parallel with nvcc for
``-gencode arch=compute_103a,code=sm_103a`` and linked into
``paper_2012_08655_gb300/libfovea.so`` (CUDA runtime linked statically, so
the library loads without a GPU). Objects go to ``paper_2012_08655_gb300/_build``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfovea.so")
# Bounds-checked variant (-DFOVEA_BOUNDS): every global store and the tensor-
# core kernels' shared-memory stores check their address against the buffer
# they belong to, record FOVEA_FAULT_BOUNDS and skip the access instead of
# writing out of bounds. A debugging aid, loaded through FOVEA_LIBRARY.
BUILD_BOUNDS = os.path.join(HERE, "_build_bounds")
LIB_BOUNDS = os.path.join(HERE, "libfovea_bounds.so")

SOURCES = ["sigma.cu", "forward.cu", "tc_forward.cu", "umma_forward.cu", "tc05_forward.cu", "tcf_forward.cu", "tca_adjoint.cu", "pixel_forward.cu", "pyramid.cu", "ssim.cu", "adjoint.cu", "noalloc.cu", "peak.cu",
           "api.cu", "tune.cpp", "server.cpp"]
HEADERS = ["fovea_internal.cuh", "fovea_host.h", "fwd_common.cuh", "tc_common.cuh", "tc05_common.cuh", "arena.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: libfovea.so cannot be built")


def _flags(extra=()):
    return ["-O3", "-std=c++17", "-lineinfo", "-I", INCLUDE, "-I", CSRC,
            "-Xcompiler", "-fPIC,-ffp-contract=off", *ARCH, *extra]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=(), bounds: bool = False) -> str:
    """Compile (if out of date) and return the path of libfovea.so (or, with
    ``bounds``, of the bounds-checked libfovea_bounds.so)."""
    nvcc = _nvcc()
    build_dir, lib = (BUILD_BOUNDS, LIB_BOUNDS) if bounds else (BUILD, LIB)
    if bounds:
        extra_flags = (*extra_flags, "-DFOVEA_BOUNDS")
    os.makedirs(build_dir, exist_ok=True)
    common = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "fovea.h")]
    procs, objs = [], []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(build_dir, src + ".o")
        objs.append(obj)
        if force or _stale(obj, [path, *common, __file__]):
            cmd = [nvcc, *_flags(extra_flags), "-c", path, "-o", obj]
            if src.endswith(".cpp"):
                cmd = [nvcc, "-x", "c++", *_flags(extra_flags), "-c", path, "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            sys.stderr.write(out.decode(errors="replace"))
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError(f"libfovea build failed:\n{msg}")
    if force or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, bounds="--bounds" in sys.argv))
