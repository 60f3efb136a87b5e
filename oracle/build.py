"""Build the FP64 oracle's shared library (test infrastructure) with g++.

The library is written next to this file as `liborc.so`.  It is rebuilt when any source is
newer than the library.  Generic x86-64 code (no -march=native) so the library built on one
host also runs on another.  The timed CPU legs (the bench's CPU baseline and reference arm)
use `liborc_native.so`, the same sources at -O3 -march=native, built on the host that runs them.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["orc_model.cpp", "orc_capi.cpp"]
HEADERS = ["orc_math.hpp", "orc_model.hpp", "orc_step.hpp", "orc_ad.hpp", "orc_count.hpp"]
LIB = os.path.join(HERE, "liborc.so")
LIB_NATIVE = os.path.join(HERE, "liborc_native.so")


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(os.path.join(HERE, f)) > t for f in SOURCES + HEADERS)


def build(force: bool = False, native: bool = False) -> str:
    lib = LIB_NATIVE if native else LIB
    if force or needs_build(lib):
        tmp = lib + ".%d.tmp" % os.getpid()
        opt = ["-O3", "-march=native"] if native else ["-O2"]
        cmd = ["g++", *opt, "-std=c++17", "-shared", "-fPIC", "-pthread", "-Wall", "-Wno-unused-function",
               "-o", tmp] + [os.path.join(HERE, s) for s in SOURCES]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
