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
            ("adjoint_body.cuh", os.path.join(CSRC, "adjoint_body.cuh")),
            ("branch_body.cuh", os.path.join(CSRC, "branch_body.cuh"))]
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
    return any(os.path.getmtime(f) > t for f in sources() + _headers())


# headers that only the run-time compiler sees (embedded, included by no source compiled here)
RTC_ONLY = {"branch_body.cuh"}


def _headers(compiled_only: bool = False):
    hs = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return [h for h in hs if not (compiled_only and os.path.basename(h) in RTC_ONLY)]


def _object(src: str) -> str:
    return os.path.join(BUILD_DIR, os.path.basename(src) + ".o")


def compile_cmd(src: str, out: str, verbose: bool = False):
    cmd = ["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-c", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
           "-o", out, src]
    if verbose:
        cmd[1:1] = ["-Xptxas", "-v"]
    return cmd


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every source to an object under _build/ (in parallel, each only when it or a
    header is newer than its object), then link libpg.so."""
    if not (force or needs_build()):
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    write_embedded()
    newest_header = max(os.path.getmtime(f) for f in _headers(compiled_only=True))
    srcs = sources() + [EMBED_CPP]
    todo = []
    for src in srcs:
        obj = _object(src)
        if force or src == EMBED_CPP or not os.path.exists(obj) or \
                os.path.getmtime(obj) < max(os.path.getmtime(src), newest_header):
            todo.append(src)

    def run(src):
        tmp = _object(src) + ".%d.tmp" % os.getpid()
        r = subprocess.run(compile_cmd(src, tmp, verbose), capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, _object(src))
        return src, r

    with ThreadPoolExecutor(max_workers=max(1, min(len(todo), os.cpu_count() or 1))) as ex:
        results = list(ex.map(run, todo))
    for src, r in results:
        if verbose or r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode:
            raise subprocess.CalledProcessError(r.returncode, r.args)
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.run(["nvcc", *ARCH, "-shared", "-o", tmp, *[_object(s) for s in srcs], "-lcudart", "-ldl"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
