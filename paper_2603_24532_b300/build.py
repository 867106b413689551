"""Build libmbpt.so (CUDA, sm_103a) in-tree with nvcc.

    python -m paper_2603_24532_b300.build [--force]
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmbpt.so")
# launch shapes of the sample-evaluation kernel (threads per block, minimum resident blocks per SM) and
# batch parts (bit 0: denominator regulator, bit 1: group integrals, bit 2: sixth order); mbpt_k_iterate.cu
# is compiled once per (shape, part)
SHAPES = [(256, 2), (128, 4), (256, 1), (128, 3)]
PARTS = range(8)
# (source, object name, extra flags); the long kernel units first -- the sixth-order parts are the longest --
# so that they start as early as possible on a machine with fewer cores
UNITS = ([("mbpt_k_iterate.cu", "k_iterate_%dx%d_p%d" % (t, b, p),
           ["-DMBPT_TPB=%d" % t, "-DMBPT_MINB=%d" % b, "-DMBPT_PART=%d" % p])
          for p in sorted(PARTS, key=lambda q: -q) for (t, b) in SHAPES] +
         [(src, src, []) for src in ("mbpt_runtime.cu", "mbpt_host.cpp", "mbpt_k_misc.cu")])
SOURCES = sorted({u[0] for u in UNITS})
HEADERS = ["mbpt_device.cuh", "mbpt_kernels.cuh", "mbpt_kernels.h", "mbpt_internal.h",
           os.path.join("..", "..", "include", "mbpt.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


OBJDIR = os.path.join(HERE, "_build")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    for f in SOURCES + HEADERS:
        if os.path.getmtime(os.path.join(CSRC, f)) > t:
            return True
    return False


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the translation units in parallel (the kernel shapes and batch parts are separate units)
    and link.  Objects are kept in _build/: a unit is recompiled when it, or any header, is newer than
    its object (or with force)."""
    if not force and not _stale():
        return LIB
    import concurrent.futures
    os.makedirs(OBJDIR, exist_ok=True)
    newest_header = max(os.path.getmtime(os.path.join(CSRC, h)) for h in HEADERS)

    def compile_one(unit):
        src, name, flags = unit
        obj = os.path.join(OBJDIR, name + ".o")
        path = os.path.join(CSRC, src)
        if (not force and os.path.exists(obj) and os.path.getmtime(obj) > os.path.getmtime(path)
                and os.path.getmtime(obj) > newest_header):
            return obj
        tmp = obj + ".tmp%d" % os.getpid()
        cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *flags, "-c", "-o", tmp, path]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.check_call(cmd)
        os.replace(tmp, obj)
        return obj

    workers = max(1, min(len(UNITS), os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
