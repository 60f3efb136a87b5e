"""The branch-parallel step kernel (pg_batch_specialize_ex with PG_SPEC_BRANCH): one thread per
(environment, branch), the trunk shared through warp shuffles, the mass matrix and the Newton
Hessian factorised as block arrowheads.  Its trajectory parity with the oracle is in
test_gpu_parity.py (the "branch" cases); here: ragged launches, joint-limit rows, status bits,
solver counters and the empty batch, each against the oracle or the thread-per-environment
kernels."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_08844_b300 import core
from paper_2502_08844_b300 import workloads as W
from tests.gpu_helpers import GpuRun, canon_qpos
from tests.test_gpu_parity import ONE_STEP_RTOL, assert_close_scaled

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("launch", ["branch", "branch-warp"])
@pytest.mark.parametrize("mname,cfg", [("quadruped", 1), ("humanoid", 3)])
@pytest.mark.parametrize("n", [1, 5, 8, 9, 37, 1500])
def test_ragged_env_counts(mname, cfg, n, launch):
    """A warp holds 32 / lanes environments and a block up to 8 warps; counts that leave a warp or a
    block partly empty (its spare groups step the last environment alongside and write nothing)."""
    m = W.model(mname)
    q0, v0 = W.initial_state(m, cfg, n)
    U = W.actions(m, cfg, n, 0, 2)
    run = GpuRun(m, n, specialize=launch)
    run.set_state(q0, v0)
    run.rollout(U, m.n_substeps)
    qg, vg, _ = run.get()
    qo, vo, _, _ = O.OracleModel(m).rollout(q0, v0, U, m.n_substeps, nthreads=8)
    for e in range(n):
        assert_close_scaled("qpos %d" % e, canon_qpos(m, qg[e]), canon_qpos(m, qo[e]), 1e-4)
        assert_close_scaled("qvel %d" % e, vg[e], vo[e], 1e-4)


def test_joint_limit_rows():
    """Quadruped states with knees and hips beyond their limits (limit rows on every lane, with
    the feet in contact) and a warm start: one control step against the oracle."""
    m = W.quadruped()
    n = 16
    q0, v0 = W.initial_state(m, 1, n)
    q0 = q0.copy()
    rng = np.random.default_rng(5)
    for e in range(n):
        q0[e, 7 + 8 + (e % 4)] = -2.72 - 0.02 * rng.random()     # a knee below its lower limit
        q0[e, 7 + 2 * (e % 4)] = 1.0 + 0.01 * rng.random()        # an abduction above its upper limit
    warm = rng.normal(size=(n, m.nv)).astype(np.float32) * 5
    run = GpuRun(m, n, specialize="branch")
    run.set_state(q0, v0, warm)
    U = W.actions(m, 1, n, 0, 1)
    run.rollout(U, m.n_substeps)
    qg, vg, _ = run.get()
    qo, vo, _, _ = O.OracleModel(m).rollout(q0, v0, U, m.n_substeps, qacc_warm=warm, nthreads=8)
    for e in range(n):
        assert_close_scaled("qpos %d" % e, canon_qpos(m, qg[e]), canon_qpos(m, qo[e]), ONE_STEP_RTOL)
        vscale = max(np.abs(vo[e]).max(), 1.0)
        assert_close_scaled("qvel %d" % e, vg[e], vo[e], ONE_STEP_RTOL, vscale)


def test_status_bits():
    m = W.quadruped()
    n = 8
    q0, v0 = W.initial_state(m, 1, n)
    q0[3, 2] = np.nan          # env 3: non-finite position
    warm = np.zeros((n, 18), np.float32)
    warm[5, 4] = np.inf        # env 5: non-finite warm start
    run = GpuRun(m, n, specialize="branch")
    run.set_state(q0, v0, warm)
    run.step(W.actions(m, 1, n, 0, 1)[0], 5)
    st = run.status()
    assert st[3] & 1
    assert st[5] & 8 and not st[5] & 1
    assert all(st[e] & 1 == 0 for e in range(n) if e != 3)


def test_solver_counters_match_thread_kernel():
    """Rows assembled per substep are a count of active contacts and limits: identical to the
    thread-per-environment kernel's; Newton iterations agree on (almost) every environment."""
    m = W.quadruped()
    n = 256
    q0, v0 = W.initial_state(m, 1, n)
    U = W.actions(m, 1, n, 0, 4)
    stats = []
    for spec in (True, "branch"):
        run = GpuRun(m, n, specialize=spec)
        run.set_state(q0, v0)
        st = run.state.enable_stats()
        run.rollout(U, 5)
        stats.append(st.cpu().numpy()[:, :n].astype(np.int64))
    assert np.array_equal(stats[0][1], stats[1][1])
    assert np.mean(stats[0][0] == stats[1][0]) >= 0.95


def test_empty_batch():
    m = W.quadruped()
    cm = core.CompiledModel(m)
    b = core.Batch([(cm, 0)])
    b.specialize(branch=True)
    st = core.State(b, "cuda")
    ctrl = torch.zeros((m.nu, st.ld), device="cuda")
    core.step(b, st, ctrl, 5)
    torch.cuda.synchronize()


def test_kernel_query_and_opt_out():
    m = W.quadruped()
    cm = core.CompiledModel(m)
    b = core.Batch([(cm, 16)])
    assert b.kernel()["kernel"] == "generic"
    b.specialize(branch=False)
    assert b.kernel()["kernel"] == "specialised"
    b2 = core.Batch([(cm, 16)])
    b2.specialize()
    k = b2.kernel()
    assert k["kernel"] == "branch-parallel" and k["lanes_per_env"] == 4 and k["branches"] == 4
    assert k["barrier_per_substep"]
    h = core.CompiledModel(W.hand())
    b3 = core.Batch([(h, 16)])
    b3.specialize()
    k = b3.kernel()
    assert k["kernel"] == "specialised" and "max_contacts" in k["reason"]


@pytest.mark.parametrize("mname,cfg,n,T,rtol", [("quadruped_rough", 1, 37, 1, ONE_STEP_RTOL),
                                                ("quadruped_rough", 1, 33, 50, 1e-3),
                                                ("humanoid_rough", 3, 33, 1, ONE_STEP_RTOL)])
def test_terrain_contacts_on_the_branch_kernel(mname, cfg, n, T, rtol):
    """The rough terrain in the branch kernel: the quadruped's sphere feet (heightfield-sphere) and
    the humanoid's box feet (heightfield against the box as a solid), against the oracle; one
    control step at the one-step tolerance, 50 steps of the quadruped at the rollout tolerance."""
    m = W.model(mname)
    q0, v0 = W.initial_state(m, cfg, n)
    U = W.actions(m, cfg, n, 0, T)
    run = GpuRun(m, n, specialize="branch")   # (asserts the branch-parallel kernel runs)
    run.set_state(q0, v0)
    run.rollout(U, m.n_substeps)
    qg, vg, _ = run.get()
    qo, vo, _, _ = O.OracleModel(m).rollout(q0, v0, U, m.n_substeps, nthreads=8)
    for e in range(n):
        assert_close_scaled("qpos %d" % e, canon_qpos(m, qg[e]), canon_qpos(m, qo[e]), rtol)
        assert_close_scaled("qvel %d" % e, vg[e], vo[e], rtol)
