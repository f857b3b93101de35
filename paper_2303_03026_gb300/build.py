"""Builds the CUDA library libamrvac_gb300.so in-tree for sm_103a.

Each translation unit is compiled in parallel with nvcc (one -gencode, no
cmake), then linked into paper_2303_03026_gb300/_lib/.  Run ``python -m
paper_2303_03026_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libamrvac_gb300.so")
SOURCES = ["api.cu", "plain.cu", "fused.cu", "noalloc.cu", "fix.cu", "reflux.cu", "regrid.cu"]
# the fused kernel source is compiled once per (precision, dimension, limiter)
# limiter groups: minmod, vanleer, koren as compile-time limiters, -1 = the
# other two-ghost-cell limiters at run time, -2 = the five-point limiters at run
# time (2D tiles only)
FUSED_GROUPS = ([(t, d, l) for t in ("float", "double") for d in (2, 3) for l in (0, 1, 2, -1)] +
                [(t, 2, -2) for t in ("float", "double")] + [("float", 3, -2)])
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
              "--expt-relaxed-constexpr"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _digest() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(ROOT, "include", "amrvac.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + [os.uname().machine]).encode())
    return h.hexdigest()


# the translation unit of the fused stage kernels and everything it includes
FUSED_KERNEL_FILES = ["fused_inst.cu", "fused.cuh", "fused2d.cuh", "ghost.cuh", "physics.cuh",
                      "physics_f2.cuh", "reduce.cuh", "state.hpp", "common.cuh"]


def kernel_digest() -> str:
    """Fingerprint of the fused stage kernels alone (their sources, the public
    header, flags and host machine): hardware counters taken on one build stay
    valid for another with the same fingerprint."""
    h = hashlib.sha256()
    for name in FUSED_KERNEL_FILES:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(ROOT, "include", "amrvac.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + [os.uname().machine]).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    stamp = os.path.join(OUT_DIR, "build.stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        if open(stamp).read().strip() == dig:
            return LIB
    nvcc = _nvcc()
    objs = []

    units = [(src, src.replace(".cu", ".o"), []) for src in SOURCES]
    for t, d, l in FUSED_GROUPS:
        # FP32 bulk: approximate single-precision division and square root
        # (MUFU based, <= 2 ulp) and flush-to-zero; double arithmetic unaffected
        fast = ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"] if t == "float" else []
        units.append(("fused_inst.cu", "fused_%s_%dd_l%s.o" % (t, d, {-1: "rt", -2: "r5"}.get(l, l)),
                      ["-DAMRVAC_FT=" + t, "-DAMRVAC_FD=%d" % d, "-DAMRVAC_FL=%d" % l] + fast))

    def compile_one(unit):
        src, objname, defs = unit
        obj = os.path.join(OUT_DIR, objname)
        cmd = [nvcc] + ARCH + NVCC_FLAGS + defs + ["-I", os.path.join(ROOT, "include"), "-c",
                                                   os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr[-6000:]))
        return obj, r.stderr

    workers = max(2, min(len(units), os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        for obj, log in ex.map(compile_one, units):
            objs.append(obj)
            if verbose:
                sys.stderr.write(log)
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr[-4000:])
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
