"""Build the FP64 oracle's shared library (test infrastructure) with g++.

The library is written next to this file as `liborc.so`.  It is rebuilt when any source is
newer than the library.  Generic x86-64 code (no -march=native) so the library built on one
host also runs on another.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["orc_model.cpp", "orc_capi.cpp"]
HEADERS = ["orc_math.hpp", "orc_model.hpp", "orc_step.hpp", "orc_ad.hpp", "orc_count.hpp"]
LIB = os.path.join(HERE, "liborc.so")


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(os.path.join(HERE, f)) > t for f in SOURCES + HEADERS)


def build(force: bool = False) -> str:
    if force or needs_build():
        tmp = LIB + ".%d.tmp" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-Wall", "-Wno-unused-function",
               "-o", tmp] + [os.path.join(HERE, s) for s in SOURCES]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
