"""Build libtsnnls.so (the CUDA library behind include/tsnnls.h) in-tree.

Every .cu file under csrc/ is compiled for sm_103a with nvcc and every .cpp
file (host-only code) with the host C++ compiler, all in parallel, and linked
into ``_build/libtsnnls.so``; the CUDA runtime is linked statically so the
library has no dependency beyond the NVIDIA kernel-mode driver.  The same
sources built with -DTSNNLS_CHECK give ``_build/libtsnnls_check.so``, whose
kernels test their data-dependent indices (the debug build of the tests).
"""
from __future__ import annotations

import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libtsnnls.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtsnnls")
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _cxx() -> str:
    return shutil.which("g++") or shutil.which("c++") or "g++"


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + [os.path.join(ROOT, "include", "tsnnls.h")])


def build_id() -> str:
    """Content hash of every source and header: names this build in the
    autotuner's cache keys, so a rebuilt kernel never reuses old timings."""
    h = hashlib.sha1()
    for p in _sources() + _headers():
        with open(p, "rb") as f:
            h.update(os.path.basename(p).encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


LIB_CHECK = os.path.join(OUT_DIR, "libtsnnls_check.so")
VARIANTS = {"normal": (LIB, OUT_DIR, []), "check": (LIB_CHECK, os.path.join(OUT_DIR, "check"), ["-DTSNNLS_CHECK"])}


def up_to_date(variant: str = "normal") -> bool:
    lib = VARIANTS[variant][0]
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _sources() + _headers() + [__file__])


def build(force: bool = False, verbose: bool = False, variants=("normal", "check")) -> str:
    """Build the requested variants (all translation units of all of them
    compiled in parallel): ``normal`` is libtsnnls.so, ``check`` the
    bounds-checked libtsnnls_check.so (-DTSNNLS_CHECK).  Returns the normal
    library's path."""
    todo = [v for v in variants if force or not up_to_date(v)]
    if not todo:
        return LIB
    nvcc = _nvcc()
    bid = "-DTSNNLS_BUILD_ID=\"" + build_id() + "\""
    procs = []
    links = []
    for v in todo:
        lib, odir, defs = VARIANTS[v]
        os.makedirs(odir, exist_ok=True)
        objs = []
        for src in _sources():
            obj = os.path.join(odir, os.path.splitext(os.path.basename(src))[0] + ".o")
            objs.append(obj)
            if src.endswith(".cpp"):
                cmd = [_cxx(), "-O2", "-std=c++17", "-fPIC", "-Wall", "-I" + os.path.join(ROOT, "include"),
                       "-I" + CSRC] + defs + ["-c", src, "-o", obj]
            else:
                cmd = [nvcc] + ARCH + NVCC_FLAGS + [bid] + defs + ["-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        links.append((lib, objs))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    for lib, objs in links:
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"], check=True)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
