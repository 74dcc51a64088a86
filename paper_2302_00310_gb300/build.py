"""In-tree build of the CUDA library ``libpond_gb300.so`` (sm_103a only).

The translation units are compiled in parallel with nvcc and linked into one
shared library next to this file.  Nothing is installed into site-packages.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpond_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpond_gb300.so")
    return cand


def _digest() -> str:
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(CSRC, "*"))) + sorted(glob.glob(os.path.join(INCLUDE, "*.h"))):
        with open(p, "rb") as fh:
            h.update(os.path.basename(p).encode() + fh.read())
    # the flags without the include directories: those are absolute paths,
    # which differ between checkouts of the same sources
    h.update(" ".join(ARCH + [f for f in FLAGS if f not in (INCLUDE, CSRC)]).encode())
    return h.hexdigest()


# the sources that make the 2D/1D step kernels of the two main translation
# units (D2Q16 f, D2Q9 g): their machine code changes only with these files
# or the flags (the batch, ABI and check sources around them do not enter it)
KERNEL_SOURCES = ("pond_hermite.cuh", "pond_packed.cuh", "pond_kernels.cuh", "pond_launch.h",
                  "pond_step_impl.cuh", "pond_step_fp64.cu", "pond_step_fp32.cu")


def kernel_digest() -> str:
    """Digest of the step kernels' sources and flags, the key under which
    counters taken on one build stay valid for another."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(CSRC, name), "rb") as fh:
            h.update(name.encode() + fh.read())
    h.update(" ".join(ARCH + [f for f in FLAGS if f not in (INCLUDE, CSRC)]).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every ``csrc/*.cu`` for sm_103a and link ``libpond_gb300.so``."""
    stamp = os.path.join(BUILD, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def comp(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s" % (src, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        results = list(ex.map(comp, srcs))
    if verbose or ptxas_info:
        for _, log in results:
            print(log)
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr)
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="-v" in sys.argv))
