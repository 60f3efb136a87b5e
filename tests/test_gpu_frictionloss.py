"""GPU parity of joint friction loss (friction-loss rows) against the FP64 oracle through the C
ABI: every phase of a substep, including the rows' Jacobian, reference acceleration, D, Ahat
and force, on a one-joint arm and on the quadruped with friction loss on its twelve hinges; one
control step and 50-step rollouts at the step tolerances; specialised against generic."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_08844_b300 import core, workloads as W
from tests.gpu_helpers import GpuRun, canon_qpos
from tests.test_gpu_parity import ONE_STEP_RTOL, ROLLOUT_RTOL, _phase_compare, assert_close_scaled

pytestmark = pytest.mark.gpu


def _quadruped_with_friction(F=0.8):
    m = W.quadruped()
    fl = np.zeros(m.nv, np.float32)
    fl[6:] = F
    m.dof_frictionloss = fl
    return m


def _arm(F=0.3):
    b = W.ModelBuilder("fric_arm")
    link = b.body(0, (0, 0, 0))
    b.joint(link, W.HINGE, axis=(0, 0, 1), frictionloss=F)
    b.geom(link, W.BOX, (0.2, 0.05, 0.05), pos=(0.2, 0, 0), mass=2.0)
    b.actuator(0, W.MOTOR, gear=1.0)
    return b.build(timestep=0.002, gravity=(0, 0, 0), iterations=4)


@pytest.mark.parametrize("v0,u", [(2.0, 0.0), (-0.5, 0.1), (0.0, 0.2), (0.01, -1.0)])
def test_phase_parity_friction_arm(v0, u):
    m = _arm()
    om = O.OracleModel(m)
    g, o = _phase_compare(m, om, np.zeros(1), np.array([v0]), np.array([u]), env=1, n=4)
    assert g["nrow"] == 1


def test_phase_parity_quadruped_with_friction_loss():
    m = _quadruped_with_friction()
    om = O.OracleModel(m)
    q0, v0 = W.initial_state(m, 1, 3)
    U = W.actions(m, 1, 3, 0, 40)
    _, _, _, _, tq, tv = om.rollout(q0, v0, U, 5, trajectory=True)
    for t, e in ((0, 0), (10, 1), (25, 2), (39, 0)):
        g, o = _phase_compare(m, om, tq[t, e].astype(np.float32).astype(np.float64),
                              tv[t, e].astype(np.float32).astype(np.float64), U[t + 1 if t < 39 else t, e].astype(np.float64),
                              env=e, n=4)
        assert g["nrow"] >= 12                       # the twelve friction-loss rows at least


@pytest.mark.parametrize("n,T,rtol", [(37, 1, ONE_STEP_RTOL), (33, 50, ROLLOUT_RTOL)])
def test_quadruped_friction_loss_trajectories(n, T, rtol):
    m = _quadruped_with_friction()
    om = O.OracleModel(m)
    q0, v0 = W.initial_state(m, 1, n)
    U = W.actions(m, 1, n, 0, T)
    run = GpuRun(m, n)
    run.set_state(q0, v0)
    run.rollout(U, m.n_substeps)
    qg, vg, _ = run.get()
    qo, vo, _, _ = om.rollout(q0, v0, U, m.n_substeps, nthreads=8)
    for e in range(n):
        assert_close_scaled("qpos env %d" % e, canon_qpos(m, qg[e]), canon_qpos(m, qo[e]), rtol)
        assert_close_scaled("qvel env %d" % e, vg[e], vo[e], rtol)
    # the loss matters: without it the same steps end elsewhere
    qf, _, _, _ = O.OracleModel(W.quadruped()).rollout(q0, v0, U, m.n_substeps, nthreads=8)
    assert np.abs(qf - qo).max() > 1e-4


def test_specialised_friction_loss_matches_generic():
    import torch
    m = _quadruped_with_friction()
    outs = []
    for spec in (False, True):
        run = GpuRun(m, 128)
        if spec:
            run.batch.specialize()
        q0, v0 = W.initial_state(m, 1, 128)
        run.set_state(q0, v0)
        run.rollout(W.actions(m, 1, 128, 0, 10), 5)
        outs.append(run.get())
    for a, b in zip(outs[0], outs[1]):
        assert np.allclose(a, b, rtol=1e-4, atol=1e-5)
