"""Edge cases through the C ABI on the GPU: empty batches through every entry point, and one
control step of models at the kernels' capacity limits (64 dofs; 128 constraint rows, all four
words of the active-set masks in use) against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_08844_b300 import core, workloads as W
from tests import models_for_tests as MT
from tests.gpu_helpers import GpuRun, canon_qpos
from tests.test_gpu_parity import ONE_STEP_RTOL, assert_close_scaled

pytestmark = pytest.mark.gpu


def test_empty_batch_through_every_entry_point():
    m = W.quadruped()
    cm = core.CompiledModel(m)
    batch = core.Batch([(cm, 0)])
    assert batch.n == 0
    st = core.State(batch, "cuda")
    ld = st.ld
    ctrl = torch.zeros((m.nu, ld), device="cuda")
    core.step(batch, st, ctrl, 5)
    core.reset(batch, st, st.qpos.clone(), st.qvel.clone())
    t = core.Task(cm, W.quadruped_task())
    ts = torch.zeros((t.state_rows, ld), device="cuda")
    obs = torch.zeros((t.nobs, ld), device="cuda")
    r = torch.zeros(ld, device="cuda")
    core.env_reset(batch, t, st, ts, st.qpos, st.qvel, torch.zeros((3, ld), device="cuda"), obs)
    core.env_step(batch, t, st, ts, ctrl, torch.zeros((3, ld), device="cuda"), st.qpos, st.qvel, 5, obs, r, r.clone(),
                  r.clone())
    core.render(batch, st, W.quadruped_scene(8, 8), torch.zeros((0, 8, 8, 3), dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()


def _limit_state(m, n, seed):
    q0 = np.tile(np.r_[0, 0, 2.0, 1, 0, 0, 0, np.zeros(m.nq - 7)], (n, 1)).astype(np.float32)
    q0[:, 7:] = np.random.default_rng(seed).uniform(-0.3, 0.3, (n, m.nq - 7))
    v0 = np.random.default_rng(seed + 1).uniform(-1, 1, (n, m.nv)).astype(np.float32)
    return q0, v0


@pytest.mark.parametrize("model", ["star", "chain"])
def test_64_dof_models_solve_their_equations_of_motion(model):
    """64 dofs, the kernels' limit, one substep.  The tree's depth sets M's conditioning: the star
    (depth 1, cond(M) ~ 3e4) and the 58-link chain (depth 59, cond(M) ~ 4e6).  In float32 the
    acceleration's forward error can reach cond(M) x 6e-8, so the check is backward error: the
    GPU's acceleration, read off v1 = v0 + h a, must satisfy the oracle's equations of motion
    M a + c(q, v) = -damping v to 1e-5 of their scale, and its positions must be the oracle's
    integration of its own velocity to the one-step tolerance.  The well-conditioned star must
    also match the oracle's step itself at the one-step tolerance."""
    m = MT.floating_star(64) if model == "star" else MT.floating_chain(64)
    n = 37
    q0, v0 = _limit_state(m, n, 0)
    om = O.OracleModel(m)
    U = np.zeros((1, n, 0), np.float32)
    run = GpuRun(m, n)
    run.set_state(q0, v0)
    run.rollout(U, 1)
    qg, vg, _ = run.get()
    qo, vo, _, _ = om.rollout(q0, v0, U, 1)
    h = float(np.float32(m.timestep))
    damping = m.dof_damping.astype(np.float64)
    for e in range(n):
        q, v = q0[e].astype(np.float64), v0[e].astype(np.float64)
        assert_close_scaled("qpos env %d (integration of its velocity)" % e, canon_qpos(m, qg[e]),
                            canon_qpos(m, om.integrate_pos(q, vg[e], h)), ONE_STEP_RTOL)
        if model == "star":
            assert_close_scaled("qpos env %d" % e, canon_qpos(m, qg[e]), canon_qpos(m, qo[e]), ONE_STEP_RTOL)
            assert_close_scaled("qvel env %d" % e, vg[e], vo[e], ONE_STEP_RTOL, max(np.abs(vo[e]).max(), 1.0))
        a = (vg[e] - v) / h
        tau = om.inverse_dynamics(q, v, a)                 # M a + c
        M = om.mass_matrix(q)
        scale = np.abs(M).max() * np.abs(a).max() + np.abs(om.inverse_dynamics(q, v, np.zeros(m.nv))).max()
        assert np.abs(tau + damping * v).max() <= 1e-5 * scale, (e, np.abs(tau + damping * v).max() / scale)


def test_128_row_model_matches_oracle():
    """32 simultaneous contacts of a plate on 33 sphere feet: 128 rows, the kernels' limit (all
    four words of the active-set masks in use), one control step at the step tolerance."""
    m = MT.many_feet(33, max_contacts=32)
    n = 33
    q0 = np.tile(m.qpos_init, (n, 1)).astype(np.float32)
    q0[:, 2] -= np.linspace(0.0, 0.004, n).astype(np.float32)    # every foot pressed into the plane
    v0 = np.zeros((n, m.nv), np.float32)
    v0[:, 3:6] = np.random.default_rng(2).uniform(-0.2, 0.2, (n, 3))
    om = O.OracleModel(m)
    f = om.forward(q0[0].astype(np.float64), v0[0].astype(np.float64))
    assert f["nrow"] == 128              # every row of the limit exists
    U = np.zeros((1, n, 0), np.float32)
    run = GpuRun(m, n)
    run.set_state(q0, v0)
    run.rollout(U, 2)
    qg, vg, _ = run.get()
    qo, vo, _, _ = om.rollout(q0, v0, U, 2)
    for e in range(n):
        assert_close_scaled("qpos env %d" % e, canon_qpos(m, qg[e]), canon_qpos(m, qo[e]), ONE_STEP_RTOL)
        assert_close_scaled("qvel env %d" % e, vg[e], vo[e], ONE_STEP_RTOL, max(np.abs(vo[e]).max(), 1.0))
