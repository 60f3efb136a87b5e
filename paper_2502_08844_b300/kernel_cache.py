"""Ahead-of-time compiles of the run-time specialised kernels (pg_model_precompile).

Batch.specialize compiles its kernels with NVRTC on first use: from a few seconds (cartpole) to
over a minute (the humanoid, the hand) per model, one model after the other.  A program that is
about to specialise many models (a test suite, the benchmark) can instead compile them all up
front, in parallel host threads and without any device work, into the disk cache (or into
kernel_cache/ beside the library file, for a build that ships its kernels); pg_batch_specialize
reads both before compiling anything itself.  The cubins are named by the same key (generated
source, NVRTC version, embedded kernel headers), so the kernels that run are the ones a run-time
compile would have produced.
"""
from __future__ import annotations

import hashlib
import os
import pickle
import time
from concurrent.futures import ThreadPoolExecutor
from typing import Iterable, List, Optional, Tuple

from . import core
from . import workloads as W

SHIPPED_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "kernel_cache")

# (model, environments, envs_per_cta as the batch is compiled with, branch-parallel kernel wanted)
Request = Tuple[W.Model, int, int, bool]


def _model_key(m: W.Model) -> str:
    return hashlib.sha1(pickle.dumps(m)).hexdigest()


def precompile(requests: Iterable[Request], cache_dir: Optional[str] = None, jobs: Optional[int] = None,
               budget_s: Optional[float] = None) -> dict:
    """Compile the kernels of every request into cache_dir (None: the disk cache that
    pg_batch_specialize writes; SHIPPED_DIR: kernel_cache/ beside the library, for a build that
    ships its kernels).  One task per distinct (model, environments per warp): its
    thread-per-environment cubin, and for the model's first task the branch-parallel cubin when
    any request asks for it; so no two tasks compile the same source.  The costliest models (most
    degrees of freedom, the elliptic cone) start first, on `jobs` threads (default: the host's
    cores).  Tasks not started within budget_s seconds are skipped (their kernels compile at run
    time as before).  Returns counts and the wall time."""
    t0 = time.time()
    failed: List[str] = []
    models = {}
    for m, count, epc, branch in requests:
        models.setdefault(_model_key(m), (m, []))[1].append((int(count), int(epc), bool(branch)))
    tasks = []
    for m, reqs in models.values():
        try:
            cm = core.CompiledModel(m)
            widths = {}
            for count, epc, _ in reqs:
                widths.setdefault(cm.envs_per_warp(count, epc), (count, epc))
        except Exception as e:   # the batch compiles this model at run time instead
            failed.append("%s: %s" % (m.name, str(e).splitlines()[0] if str(e) else type(e).__name__))
            continue
        branch = any(b for _, _, b in reqs)
        for i, (count, epc) in enumerate(widths.values()):
            tasks.append((cm, count, epc, branch and i == 0))
    tasks.sort(key=lambda t: -(t[0].src.nv * (2 if t[0].src.cone == W.ELLIPTIC else 1)))

    def task(t) -> str:
        cm, count, epc, branch = t
        if budget_s is not None and time.time() - t0 > budget_s:
            return "skipped"
        try:
            cm.precompile(count, envs_per_cta=epc, branch=branch, cache_dir=cache_dir)
            return "ok"
        except Exception as e:
            return "%s: %s" % (cm.src.name, str(e).splitlines()[0] if str(e) else type(e).__name__)

    results = []
    if tasks:
        with ThreadPoolExecutor(max_workers=max(1, min(len(tasks), jobs or os.cpu_count() or 1))) as ex:
            results = list(ex.map(task, tasks))
    failed += [r for r in results if r not in ("ok", "skipped")]
    return {"models": len(models), "tasks": len(tasks), "failed": failed, "skipped": results.count("skipped"),
            "wall_s": time.time() - t0}
