"""Build the CUDA library ``libgb300rbt.so`` for sm_103a with nvcc, in tree.

Each ``csrc/*.cu`` compiles to its own object in parallel (``batched_kernels.cu``
to one object per working precision and variant of the batched solver), then
nvcc links them into ``paper_2312_09376_gb300/_build/libgb300rbt.so``
(git-ignored).  The build is skipped when the library is newer than every
source and header.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgb300rbt.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")]
# batched_kernels.cu holds a whole solver (and its adjoint) per working
# precision and variant inside persistent kernels: one object per
# instantiation, so that NVVM optimises each at its full level and the eight
# compile side by side (all in one object, about twenty minutes).
MULTI = {"batched_kernels.cu": [("batched_kernels_%s_%d_%d" % ("f64" if p == 0 else "f32", nt, nb),
                                 ["-DRBT_BAT_PREC=%d" % p, "-DRBT_BAT_NT=%d" % nt, "-DRBT_BAT_NB=%d" % nb])
                                for p in (1, 0) for nt, nb in ((256, 32), (128, 32), (256, 16), (128, 16))]}


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgb300rbt.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    flags = FLAGS + list(extra_flags or [])

    def compile_one(unit):
        src, name, extra = unit
        obj = os.path.join(BUILD, name + ".o")
        cmd = [nvcc] + ARCH + flags + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s %s:\n%s\n%s" % (src, " ".join(extra), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    # the slowest translation units first, so that they overlap all the others
    units = []
    for src in _sources():
        base = os.path.basename(src)
        units += [(src, name, extra) for name, extra in MULTI[base]] if base in MULTI else [(src, base[:-3], [])]
    units.sort(key=lambda u: os.path.basename(u[0]) not in MULTI)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(units), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcuda"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
