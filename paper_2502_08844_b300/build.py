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


# headers compiled again at run time by pg_batch_specialize (NVRTC), embedded in the library
EMBEDDED = [("pg.h", os.path.join(INCLUDE, "pg.h")), ("pg_internal.h", os.path.join(CSRC, "pg_internal.h")),
            ("step_device.cuh", os.path.join(CSRC, "step_device.cuh")),
            ("env_device.cuh", os.path.join(CSRC, "env_device.cuh")),
            ("step_kernel_body.cuh", os.path.join(CSRC, "step_kernel_body.cuh")),
            ("adjoint_body.cuh", os.path.join(CSRC, "adjoint_body.cuh"))]
BUILD_DIR = os.path.join(HERE, "_build")
EMBED_CPP = os.path.join(BUILD_DIR, "pg_embedded.cpp")


def write_embedded() -> str:
    """C++ source holding the embedded headers as raw string literals (regenerated every build)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    out = ["// generated by build.py from the kernel headers; do not edit", "namespace pg {",
           "extern const int kEmbeddedCount = %d;" % len(EMBEDDED),
           "extern const char* const kEmbeddedNames[] = {%s};" % ", ".join('"%s"' % n for n, _ in EMBEDDED),
           "extern const char* const kEmbeddedTexts[] = {"]
    for _, path in EMBEDDED:
        text = open(path).read()
        assert ")PGSRC\"" not in text
        out.append('R"PGSRC(' + text + ')PGSRC",')
    out += ["};", "}  // namespace pg", ""]
    tmp = EMBED_CPP + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        f.write("\n".join(out))
    os.replace(tmp, EMBED_CPP)
    return EMBED_CPP


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
           "-o", out, *sources(), EMBED_CPP, "-lcudart", "-ldl"]
    if verbose:
        cmd[1:1] = ["-Xptxas", "-v"]
    return cmd


def build(force: bool = False, verbose: bool = False) -> str:
    if force or needs_build():
        tmp = LIB + ".%d.tmp" % os.getpid()
        write_embedded()
        subprocess.run(nvcc_cmd(tmp, verbose), check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
