"""CPU checks of the ahead-of-time kernel compiles (pg_model_precompile, kernel_cache) and of the
environments-per-warp rule that pg_batch_compile applies (no device needed for either)."""
import os

import pytest

from paper_2502_08844_b300 import _capi, core, kernel_cache
from paper_2502_08844_b300 import workloads as W


@pytest.mark.parametrize("name,count,epc,want", [
    # the widest width whose warp of workspaces fits shared memory, while one wave holds them
    ("quadruped", 8192, 0, 32), ("cartpole", 8192, 0, 32), ("humanoid", 2048, 0, 16), ("hand", 64, 0, 16),
    # 8192 hands at 16 a warp need more than one wave: the width whose block holds the most of them
    ("hand", 8192, 0, 4), ("hand_elliptic", 8192, 0, 4),
    # a fixed envs_per_cta keeps the widest width
    ("hand", 8192, 16, 16),
])
def test_envs_per_warp_rule(name, count, epc, want):
    assert core.CompiledModel(W.model(name)).envs_per_warp(count, epc) == want


def test_envs_per_warp_depends_on_the_multiprocessor_count():
    hand = core.CompiledModel(W.model("hand"))
    # 2000 SMs hold 8192 hands in one wave at the widest width
    assert hand.envs_per_warp(8192, sms=2000) == 16
    assert hand.envs_per_warp(8192, sms=0) == hand.envs_per_warp(8192, sms=148)


def test_precompile_rejects_bad_arguments():
    cm = core.CompiledModel(W.model("cartpole"))
    for args in ((-1, 0, 0, 0), (8, -1, 0, 0), (8, 257, 0, 0), (8, 0, -1, 0), (8, 0, 0, 64)):
        with pytest.raises(_capi.PgError) as e:
            _capi.pg_model_precompile(cm.handle, *args, None)
        assert e.value.code == _capi.PG_EINVAL
    with pytest.raises(_capi.PgError):
        _capi.pg_model_precompile(None, 8, 0, 0, 0, None)


def test_precompile_writes_each_cubin_once(tmp_path):
    """The cartpole (no branch-parallel plan: a chain without a trunk) needs one cubin; a second
    request for it, from another count at the same width, compiles nothing."""
    cm = core.CompiledModel(W.model("cartpole"))
    assert not cm.branch_plan()["branch"]
    d = str(tmp_path / "kc")
    assert cm.precompile(256, cache_dir=d) == 32
    files = sorted(os.listdir(d))
    assert len(files) == 1 and files[0].endswith(".cubin") and os.path.getsize(os.path.join(d, files[0])) > 0
    mtime = os.path.getmtime(os.path.join(d, files[0]))
    cm.precompile(4096, cache_dir=d)
    assert sorted(os.listdir(d)) == files and os.path.getmtime(os.path.join(d, files[0])) == mtime
    # the same model through kernel_cache: one task, no new cubin
    r = kernel_cache.precompile([(W.model("cartpole"), 256, 0, True), (W.model("cartpole"), 64, 8, False)],
                                cache_dir=d)
    assert r["models"] == 1 and not r["failed"] and sorted(os.listdir(d)) == files


def test_recorder_finds_the_models_gpu_tests_specialise():
    """tests/kernel_requests.py on one GPU test file: its quadruped and humanoid batches, with
    their counts."""
    from tests.kernel_requests import collect
    reqs = collect([os.path.join(os.path.dirname(__file__), "test_gpu_branch.py")])
    names = {m.name for m, _, _, _ in reqs}
    assert {"quadruped", "humanoid"} <= names
    assert all(isinstance(n, int) and n >= 0 and isinstance(b, bool) for _, n, _, b in reqs)
