"""GPU parity of joint friction loss (friction-loss rows) against the FP64 oracle through the C
ABI: every phase of a substep, including the rows' Jacobian, reference acceleration, D, Ahat
and force, on a one-joint arm, on the quadruped with friction loss on its twelve hinges and on
the elliptic-cone hand with friction loss on its sixteen (App. C.2.2); one control step and
rollouts at the step tolerances; specialised against generic."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_08844_b300 import core, workloads as W
from tests.gpu_helpers import GpuRun, canon_qpos
from tests.test_gpu_parity import ONE_STEP_RTOL, ROLLOUT_RTOL, _phase_compare, _rollout_states, assert_close_scaled

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


# The elliptic hand with friction loss on every hinge: a tenth of the servo's maximum torque
# (App. C.2.2), taken as 0.05 N m for the hand's 3 N m/rad PD servos
HAND_FRICTIONLOSS = 0.05


def _elliptic_hand_with_friction():
    return W.hand(cone=W.ELLIPTIC, frictionloss=HAND_FRICTIONLOSS)


def test_phase_parity_elliptic_hand_with_friction_loss():
    """Elliptic contacts and friction-loss rows in one solve: every phase, the rows and their
    forces, on states along a grasp."""
    m = _elliptic_hand_with_friction()
    om, states = _rollout_states(m, 2, (0, 6, 30))
    nrows = []
    for q, v, u in states:
        g, o = _phase_compare(m, om, q, v, u, env=1, n=4)
        nrows.append(g["nrow"])
    assert min(nrows) >= 16                          # the sixteen friction-loss rows at least
    assert max(nrows) >= 16 + 6                      # and elliptic contacts


@pytest.mark.parametrize("specialize", [pytest.param(False, id="generic"), pytest.param(True, id="specialised")])
def test_elliptic_hand_with_friction_loss_one_step_and_reanchored(specialize):
    """One control step on 40 environments at the one-step tolerance, then 20 more steps on 16 of
    them, each compared with the oracle's step from the GPU's own state (re-anchored, as the
    elliptic hand's long rollouts are).  qvel's scale is the larger of |qvel| and the step's
    velocity change: friction loss holds joints nearly still (|qvel| small) while the substeps'
    h qacc terms, whose FP32 rounding reaches qvel, stay as large as without it."""
    m = _elliptic_hand_with_friction()
    om = O.OracleModel(m)
    n = 40
    q0, v0 = W.initial_state(m, 2, n)
    U = W.actions(m, 2, n, 0, 21)
    run = GpuRun(m, n, specialize=specialize)
    run.set_state(q0, v0)
    q, v, w = q0.astype(np.float64), v0.astype(np.float64), np.zeros((n, m.nv))
    for t in range(21):
        run.step(U[t], m.n_substeps)
        qg, vg, wg = run.get()
        qo, vo, _, _ = om.rollout(q, v, U[t:t + 1], m.n_substeps, qacc_warm=w, nthreads=8)
        for e in range(n if t == 0 else 16):
            assert_close_scaled("step %d qpos env %d" % (t, e), canon_qpos(m, qg[e]), canon_qpos(m, qo[e]), ONE_STEP_RTOL)
            vscale = max(np.abs(vo[e]).max(), np.abs(vo[e] - v[e]).max())
            assert_close_scaled("step %d qvel env %d" % (t, e), vg[e], vo[e], ONE_STEP_RTOL, scale=vscale)
        q, v, w = qg, vg, wg
    # the loss matters: without it the first step already ends elsewhere
    qf, _, _, _ = O.OracleModel(W.hand_elliptic()).rollout(q0, v0, U[:1], m.n_substeps, nthreads=8)
    qo1, _, _, _ = om.rollout(q0, v0, U[:1], m.n_substeps, nthreads=8)
    assert np.abs(qf - qo1).max() > 1e-5
