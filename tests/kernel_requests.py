"""Which models the GPU tests specialise, found without a GPU, so that their kernels can be
compiled in parallel before the first test (paper_2502_08844_b300.kernel_cache).

`collect()` runs the GPU tests once in a child pytest, on the CPU and with no device visible,
with this module as a plugin.  The plugin replaces core.Batch by a recorder: each batch a test
builds is recorded (its models, environment counts and envs_per_cta) and ends the test at its
first use (or at the first use of a state made for it), so no test computes anything.  A test that builds a second batch after using its
first is recorded up to the first; the rest of its kernels compile at run time as before.
"""
from __future__ import annotations

import inspect
import os
import pickle
import subprocess
import sys
import tempfile
from typing import List

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHILD_ENV = "PG_KERNEL_REQUESTS_OUT"

_records = []
_current = {"mentions_specialize": False}


class _Recorded(Exception):
    pass


def pytest_configure(config):
    if not os.environ.get(CHILD_ENV):
        return
    import torch
    from paper_2502_08844_b300 import core

    class RecordingBatch:
        def __init__(self, parts, envs_per_cta: int = 0):
            parts = list(parts)
            self.rec = {"parts": [(cm.src, int(n)) for cm, n in parts], "epc": int(envs_per_cta), "branch": None,
                        "mentions_specialize": _current["mentions_specialize"]}
            _records.append(self.rec)

        def specialize(self, branch: bool = True, warp_blocks: bool = False):
            self.rec["branch"] = bool(branch or warp_blocks)
            raise _Recorded()

        def __getattr__(self, name):
            raise _Recorded()

    class InertState:
        """A state that can be made but not used: tests that build their state before they
        specialise the batch (GpuRun) still reach the specialisation."""

        def __init__(self, *args, **kwargs):
            pass

        def __getattr__(self, name):
            raise _Recorded()

    core.Batch = RecordingBatch
    core.State = InertState
    # the GPU tests' fixture asks torch for a device; the recorder stops each test before it
    # touches one
    torch.cuda.is_available = lambda: True


def pytest_runtest_setup(item):
    """Whether the test's own source mentions specialisation: a test that compares the generic
    kernel with a specialised one often builds the generic batch first, and the recording stops
    there."""
    try:
        _current["mentions_specialize"] = "specialize" in inspect.getsource(item.function)
    except (AttributeError, OSError, TypeError):
        _current["mentions_specialize"] = False


def pytest_sessionfinish(session, exitstatus):
    out = os.environ.get(CHILD_ENV)
    if out:
        with open(out, "wb") as f:
            pickle.dump(_records, f)


def collect(test_paths: List[str], timeout_s: float = 300.0) -> list:
    """kernel_cache requests (model, count, envs_per_cta, branch) of the GPU tests under
    test_paths: the batches that the recording saw specialised, and the batches of tests whose
    source mentions specialisation where the recording stopped first (with the branch-parallel
    kernel, which compiles only for a model that qualifies).  Batches of other tests run the
    library's generic kernel and need no compile."""
    with tempfile.TemporaryDirectory() as tmp:
        out = os.path.join(tmp, "requests.pkl")
        env = dict(os.environ, CUDA_VISIBLE_DEVICES="", **{CHILD_ENV: out})
        env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
        subprocess.run([sys.executable, "-m", "pytest", *test_paths, "-m", "gpu", "-q", "-p", "tests.kernel_requests",
                        "-p", "no:cacheprovider", "--no-header", "-o", "addopts="],
                       cwd=ROOT, env=env, stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL, timeout=timeout_s)
        with open(out, "rb") as f:
            records = pickle.load(f)
    reqs = []
    for r in records:
        if r["branch"] is not None:
            reqs += [(m, n, r["epc"], r["branch"]) for m, n in r["parts"]]
        elif r["mentions_specialize"]:
            reqs += [(m, n, r["epc"], True) for m, n in r["parts"]]
    return reqs
