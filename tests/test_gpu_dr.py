"""GPU parity of per-environment parameters (pg_step_dr) and actuator torque limits against the
FP64 oracle through the C ABI.  An environment with parameters p must move as the oracle's
substituted model (oracle/randomize.py) does; the tolerances are the step's own (one control
step 1e-5 of each vector's scale, 1e-6 absolute; 20-step rollouts 1e-3)."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import randomize as RZ
from paper_2502_08844_b300 import core, workloads as W
from tests.gpu_helpers import GpuRun, canon_qpos
from tests.test_gpu_parity import ONE_STEP_RTOL, ROLLOUT_RTOL, assert_close_scaled

pytestmark = pytest.mark.gpu


def _run_dr(m, q0, v0, U, P, T, specialize=False):
    """specialize: False (generic), True (the specialised thread-per-environment kernel) or
    "branch" (the branch-parallel kernel's per-environment-parameter variant)"""
    run = GpuRun(m, q0.shape[0])
    if specialize:
        run.batch.specialize(branch=specialize == "branch")
        if specialize == "branch":
            k = run.batch.kernel()
            assert k["kernel"] == "branch-parallel" and k["branch_dr"]
    run.set_state(q0, v0)
    params = torch.from_numpy(core.to_soa(P, run.state.ld, P.shape[1])).to("cuda")
    for t in range(T):
        core.step_dr(run.batch, run.state, run.ctrl_tensor(U[t]), params, m.n_substeps)
    return run.get()


def _oracle_env(m, q0, v0, U, p, T):
    mz = RZ.substituted_model(m, p.astype(np.float64))
    q, v, _, _ = O.OracleModel(mz).rollout(q0[None], v0[None], RZ.controls(m, p, U[:T]), m.n_substeps)
    return q[0], v[0]


@pytest.mark.parametrize("specialize", [pytest.param(False, id="generic"), pytest.param("branch", id="branch")])
@pytest.mark.parametrize("T,rtol", [(1, ONE_STEP_RTOL), (20, ROLLOUT_RTOL)])
def test_step_dr_matches_the_substituted_oracle(T, rtol, specialize):
    """each environment against the oracle's substituted model: the generic kernel, and the
    branch-parallel kernel's variant (masses, inertias, centres of mass, payload, armature,
    calibration, gain scales and friction scale read per environment)"""
    m = W.quadruped()
    n = 24
    q0, v0 = W.initial_state(m, 1, n)
    U = W.actions(m, 1, n, 0, T)
    P = W.randomized_params(m, 1, n)
    qg, vg, _ = _run_dr(m, q0, v0, U, P, T, specialize=specialize)
    for e in range(n):
        qo, vo = _oracle_env(m, q0[e], v0[e], U[:, e:e + 1], P[e], T)
        assert_close_scaled("qpos env %d" % e, canon_qpos(m, qg[e]), canon_qpos(m, qo), rtol)
        assert_close_scaled("qvel env %d" % e, vg[e], vo, rtol)


def test_nominal_parameters_equal_the_plain_step():
    m = W.quadruped()
    n = 64
    q0, v0 = W.initial_state(m, 1, n)
    U = W.actions(m, 1, n, 0, 5)
    P = np.zeros((n, RZ.nrand(m)), np.float32); P[:, 0] = 1.0
    qd, vd, _ = _run_dr(m, q0, v0, U, P, 5)
    run = GpuRun(m, n)
    run.set_state(q0, v0)
    run.rollout(U, m.n_substeps)
    qp, vp, _ = run.get()
    assert np.array_equal(qd, qp) and np.array_equal(vd, vp)


def test_specialised_step_dr_matches_generic():
    """the specialised thread-per-environment kernel against the generic one (the same code)"""
    m = W.quadruped()
    n = 96
    q0, v0 = W.initial_state(m, 1, n)
    U = W.actions(m, 1, n, 0, 8)
    P = W.randomized_params(m, 1, n)
    a = _run_dr(m, q0, v0, U, P, 8)
    b = _run_dr(m, q0, v0, U, P, 8, specialize=True)
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=1e-4, atol=1e-5)


def _torque_limited_quadruped():
    m = W.quadruped()
    m.act_forcelimited = np.ones(m.nu, np.int32)
    m.act_forcerange = np.tile(np.array([[-4.0, 4.0]], np.float32), (m.nu, 1))
    return m


@pytest.mark.parametrize("T,rtol", [(1, ONE_STEP_RTOL), (20, ROLLOUT_RTOL)])
def test_torque_limits_match_oracle(T, rtol):
    """The quadruped with 4 Nm torque limits: its PD errors of up to 0.3 rad at kp 35 saturate."""
    m = _torque_limited_quadruped()
    n = 24
    q0, v0 = W.initial_state(m, 1, n)
    U = W.actions(m, 1, n, 0, T)
    run = GpuRun(m, n)
    run.set_state(q0, v0)
    run.rollout(U, m.n_substeps)
    qg, vg, _ = run.get()
    qo, vo, _, _ = O.OracleModel(m).rollout(q0, v0, U, m.n_substeps)
    for e in range(n):
        assert_close_scaled("qpos env %d" % e, canon_qpos(m, qg[e]), canon_qpos(m, qo[e]), rtol)
        assert_close_scaled("qvel env %d" % e, vg[e], vo[e], rtol)
    # the limits bind: without them the same step ends elsewhere
    qf, _, _, _ = O.OracleModel(W.quadruped()).rollout(q0, v0, U, m.n_substeps)
    assert np.abs(qf - qo).max() > 1e-3


def test_step_dr_argument_errors():
    from paper_2502_08844_b300 import _capi
    m = W.quadruped()
    run = GpuRun(m, 8)
    rc = _capi._lib.pg_step_dr(run.batch.handle, run.state.c(), run.ctrl_tensor(np.zeros((8, 12))).data_ptr(),
                               None, 5, None)
    assert rc == _capi.PG_EINVAL


@pytest.mark.parametrize("specialize", [False, True])
def test_step_dr_elliptic_hand_with_friction_loss(specialize):
    """The hand's randomisation (App. C.2): PD gains, link masses and motor friction (friction-loss
    scales) beside the locomotion set, on the elliptic hand with friction loss on its sixteen
    hinges, one control step against each environment's substituted oracle model."""
    m = W.hand(cone=W.ELLIPTIC, frictionloss=0.05)
    n = 24
    q0, v0 = W.initial_state(m, 2, n)
    U = W.actions(m, 2, n, 0, 1)
    P = W.randomized_params(m, 2, n)
    R = RZ.rows(m)
    qg, vg, _ = _run_dr(m, q0, v0, U, P, 1, specialize=specialize)
    for e in range(n):
        qo, vo = _oracle_env(m, q0[e], v0[e], U[:, e:e + 1], P[e], 1)
        assert_close_scaled("qpos env %d" % e, canon_qpos(m, qg[e]), canon_qpos(m, qo), ONE_STEP_RTOL)
        assert_close_scaled("qvel env %d" % e, vg[e], vo, ONE_STEP_RTOL)
    # the new groups matter: with them zeroed the oracle ends elsewhere
    P0 = P.copy(); P0[:, R["kp"]:] = 0.0
    moved = max(np.abs(_oracle_env(m, q0[e], v0[e], U[:, e:e + 1], P0[e], 1)[0]
                       - _oracle_env(m, q0[e], v0[e], U[:, e:e + 1], P[e], 1)[0]).max() for e in range(4))
    assert moved > 1e-5


def test_branch_dr_with_nominal_parameters_follows_the_branch_step():
    """the branch kernel's per-environment-parameter variant with nominal parameters (unit scales,
    zero offsets) against the plain branch step: the same arithmetic up to contraction order"""
    m = W.quadruped_rough()
    n = 96
    q0, v0 = W.initial_state(m, 1, n)
    U = W.actions(m, 1, n, 0, 2)
    P = np.zeros((n, RZ.nrand(m)), np.float32); P[:, 0] = 1.0
    qd, vd, _ = _run_dr(m, q0, v0, U, P, 2, specialize="branch")
    run = GpuRun(m, n)
    run.batch.specialize()
    run.set_state(q0, v0)
    run.rollout(U, m.n_substeps)
    qp, vp, _ = run.get()
    assert np.allclose(qd, qp, rtol=1e-4, atol=1e-5) and np.allclose(vd, vp, rtol=1e-4, atol=1e-4)


def test_branch_dr_on_rough_terrain_matches_the_substituted_oracle():
    """The branch kernel's parameter variant on the rough terrain (heightfield-sphere feet): one
    control step of each environment against the oracle's substituted model at the one-step
    tolerance.  The friction scale enters the terrain contacts' pyramid edges, the mass
    properties the kinematics and CRBA, and the calibration and gains the PD forces."""
    m = W.quadruped_rough()
    n = 24
    q0, v0 = W.initial_state(m, 1, n)
    U = W.actions(m, 1, n, 0, 1)
    P = W.randomized_params(m, 1, n)
    qg, vg, _ = _run_dr(m, q0, v0, U, P, 1, specialize="branch")
    for e in range(n):
        qo, vo = _oracle_env(m, q0[e], v0[e], U[:, e:e + 1], P[e], 1)
        assert_close_scaled("qpos env %d" % e, canon_qpos(m, qg[e]), canon_qpos(m, qo), ONE_STEP_RTOL)
        assert_close_scaled("qvel env %d" % e, vg[e], vo, ONE_STEP_RTOL)


def test_humanoid_dr_on_a_branch_batch_matches_the_substituted_oracle():
    """pg_step_dr on a humanoid batch specialised for the branch kernel: its parameter variant
    runs when the compiler fits it like the plain kernel, and is otherwise left out for the
    thread-per-environment kernel (pg_batch_kernel's branch_dr says which).  Either way one control
    step of each environment matches the oracle's substituted model at the one-step tolerance."""
    m = W.humanoid()
    n = 8
    q0, v0 = W.initial_state(m, 3, n)
    U = W.actions(m, 3, n, 0, 1)
    P = W.randomized_params(m, 3, n)
    run = GpuRun(m, n)
    run.batch.specialize(branch=True)
    k = run.batch.kernel()
    assert k["kernel"] == "branch-parallel", k
    run.set_state(q0, v0)
    params = torch.from_numpy(core.to_soa(P, run.state.ld, P.shape[1])).to("cuda")
    core.step_dr(run.batch, run.state, run.ctrl_tensor(U[0]), params, m.n_substeps)
    qg, vg, _ = run.get()
    for e in range(n):
        qo, vo = _oracle_env(m, q0[e], v0[e], U[:, e:e + 1], P[e], 1)
        assert_close_scaled("qpos env %d (branch_dr %s)" % (e, k["branch_dr"]), canon_qpos(m, qg[e]),
                            canon_qpos(m, qo), ONE_STEP_RTOL)
        assert_close_scaled("qvel env %d" % e, vg[e], vo, ONE_STEP_RTOL)
