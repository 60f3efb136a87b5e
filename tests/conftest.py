import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_sessionstart(session):
    """Before a GPU session's first test: compile the specialised kernels its tests will ask for,
    in parallel host threads (tests/kernel_requests.py finds them), into the disk cache that
    pg_batch_specialize reads.  Each test would otherwise compile its models' kernels on first use,
    one after the other (about a minute per model).  Set PG_NO_PRECOMPILE=1 to skip."""
    markexpr = session.config.getoption("markexpr", "") or ""
    if os.environ.get("PG_KERNEL_REQUESTS_OUT") or os.environ.get("PG_NO_PRECOMPILE") or "not gpu" in markexpr:
        return   # the recorder's own child session, or no GPU tests
    if not cuda_available():
        return
    try:
        from tests.kernel_requests import collect
        from paper_2502_08844_b300 import kernel_cache
        here = str(session.config.invocation_params.dir)   # the child runs from the repository root
        paths = [os.path.join(here, str(a)) for a in session.config.args] or [os.path.join(ROOT, "tests")]
        r = kernel_cache.precompile(collect(paths), cache_dir=None)
        print("\nkernel cache: %d models compiled or found in %.0f s%s" % (
            r["models"], r["wall_s"], ("; failed: " + "; ".join(r["failed"])) if r["failed"] else ""))
    except Exception as e:   # the tests then compile their kernels on first use
        print("\nkernel cache: precompile skipped (%s)" % e)


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def cuda():
    if not cuda_available():
        pytest.skip("no CUDA device")
    import torch
    return torch.device("cuda:0")
