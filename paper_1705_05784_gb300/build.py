"""Build libfams.so for sm_103a in-tree (paper_1705_05784_gb300/lib/).

Each translation unit compiles in parallel with nvcc; geometry.cu is built
without fused multiply-add so that its integer decisions (fracture cell
counts, matrix columns of fracture pieces) follow plain IEEE-754 rounding.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "lib")
LIB = os.path.join(OUT, "libfams.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = ["util", "geometry", "system", "coarse", "basis", "coarseop", "ilu", "solve", "solve_grid",
         "flux", "api", "server"]
NOFMA = {"geometry"}


def nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfams")
    return p


def _compile(unit, verbose):
    src = os.path.join(SRC, unit + ".cu")
    obj = os.path.join(OUT, unit + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-rdc=false", "-c", src, "-o", obj]
    if unit in NOFMA:
        cmd.insert(1, "-fmad=false")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {unit}.cu:\n{r.stderr}")
    return obj, r.stderr


def build(verbose=False, force=False):
    """Compile and link; skip when the library is newer than every source."""
    os.makedirs(OUT, exist_ok=True)
    srcs = [os.path.join(SRC, f) for f in os.listdir(SRC)]
    srcs.append(os.path.join(os.path.dirname(HERE), "include", "fams.h"))
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) > max(os.path.getmtime(s) for s in srcs)):
        return LIB
    with cf.ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
        res = list(ex.map(lambda u: _compile(u, verbose), UNITS))
    if verbose:
        for _, err in res:
            sys.stderr.write(err)
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *[o for o, _ in res], "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
