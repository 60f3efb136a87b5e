"""Build the CUDA library `libpg.so` in-tree for sm_103a (nvcc; no GPU needed).

    python -m paper_2502_08844_b300.build [--force] [--verbose]

The library is written next to this file.  It is rebuilt when a source under csrc/ or the
public header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libpg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(f) > t for f in deps)


def nvcc_cmd(out: str, verbose: bool = False):
    cmd = ["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
           "-o", out, *sources(), "-lcudart"]
    if verbose:
        cmd[1:1] = ["-Xptxas", "-v"]
    return cmd


def build(force: bool = False, verbose: bool = False) -> str:
    if force or needs_build():
        tmp = LIB + ".%d.tmp" % os.getpid()
        subprocess.run(nvcc_cmd(tmp, verbose), check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
