"""Pins of the oracle's per-environment parameters (oracle/randomize.py) and actuator torque
limits against statics, closed forms and the nominal model."""
import dataclasses

import numpy as np
import pytest

from paper_2502_08844_b300 import workloads as W
from oracle import oracle as O
from oracle import randomize as RZ


def test_nominal_parameters_reproduce_the_model():
    m = W.quadruped()
    q, v = W.initial_state(m, 1, 3)
    U = W.actions(m, 1, 3, 0, 10)
    m2 = RZ.substituted_model(m, RZ.nominal(m))
    a = O.OracleModel(m).rollout(q, v, U, 5)
    b = O.OracleModel(m2).rollout(q, v, RZ.controls(m, RZ.nominal(m), U), 5)
    for x, y in zip(a[:3], b[:3]):
        assert np.allclose(x, y, rtol=0, atol=1e-12)


def _box_on_plane():
    b = W.ModelBuilder("box")
    g0 = b.geom(0, W.PLANE, (0, 0, 0))
    box = b.body(0, (0, 0, 0.1))
    b.joint(box, W.FREE)
    g1 = b.geom(box, W.BOX, (0.2, 0.1, 0.05), mass=2.0)
    b.pair(g0, g1, friction=1.0, condim=3)
    return b.build(timestep=0.002, iterations=50)


def _settle(m, p, steps=1500):
    om = O.OracleModel(RZ.substituted_model(m, p))
    q = np.array([[0, 0, 0.05, 1, 0, 0, 0]]); v = np.zeros((1, 6))
    q, v, _, _ = om.rollout(q, v, np.zeros((steps, 1, 0)), 1, solver_cap=-1)
    return om, q[0], v[0]


def _normal_force(om, q, v):
    f = om.forward(q, v, np.zeros(6), None, solver_cap=-1)
    nv = om.nv
    rows, con = f["rows"], f["contacts"]
    # pyramid edge forces act along n + mu t (t = +-t1, +-t2): their normal parts add up
    return rows[:, nv + 6].sum()


@pytest.mark.parametrize("payload", [0.0, 1.5])
def test_payload_is_carried_by_the_contacts(payload):
    """A box resting on a plane: the contacts carry (m + payload) g at rest."""
    m = _box_on_plane()
    p = RZ.nominal(m); p[1] = payload
    om, q, v = _settle(m, p)
    assert np.abs(v).max() < 1e-6
    assert _normal_force(om, q, v) == pytest.approx((2.0 + payload) * 9.81, rel=1e-6)


def test_centre_of_mass_offset_in_the_body_frame():
    m = W.quadruped()
    p = RZ.nominal(m)
    off = np.zeros((m.nbody, 3)); off[1] = [0.03, -0.01, 0.02]; off[4] = [0.0, 0.01, -0.02]
    p[2:2 + 3 * m.nbody] = off.ravel()
    q = m.qpos_init.astype(np.float64).copy(); q[3:7] = [np.cos(0.3), 0.0, 0.0, np.sin(0.3)]
    f0 = O.OracleModel(m).forward(q, np.zeros(m.nv))
    f1 = O.OracleModel(RZ.substituted_model(m, p)).forward(q, np.zeros(m.nv))
    for b in (1, 4):
        assert np.allclose(f1["xcom"][b] - f0["xcom"][b], f0["xmat"][b] @ off[b], atol=1e-12)


def test_armature_adds_to_the_mass_matrix_diagonal():
    m = W.quadruped()
    p = RZ.nominal(m)
    arm = np.linspace(0.0, 0.02, m.nv)
    p[2 + 3 * m.nbody:2 + 3 * m.nbody + m.nv] = arm
    q = m.qpos_init.astype(np.float64)
    M0 = O.OracleModel(m).mass_matrix(q)
    M1 = O.OracleModel(RZ.substituted_model(m, p)).mass_matrix(q)
    assert np.allclose(M1 - M0, np.diag(arm), atol=1e-12)


@pytest.mark.parametrize("scale", [0.0, 1.0])
def test_friction_scale(scale):
    """A ball sliding on a plane: with friction scale 0 nothing slows it, with 1 it rolls."""
    b = W.ModelBuilder("ball")
    g0 = b.geom(0, W.PLANE, (0, 0, 0))
    ball = b.body(0, (0, 0, 0.05))
    b.joint(ball, W.FREE)
    g1 = b.geom(ball, W.SPHERE, (0.05,), mass=1.0)
    b.pair(g0, g1, friction=0.5, condim=3)
    m = b.build(timestep=0.002, iterations=50)
    p = RZ.nominal(m); p[0] = scale
    om = O.OracleModel(RZ.substituted_model(m, p))
    q = np.array([[0, 0, 0.0495, 1, 0, 0, 0]]); v = np.array([[1.0, 0, 0, 0, 0, 0]])
    q, v, _, _ = om.rollout(q, v, np.zeros((300, 1, 0)), 1, solver_cap=-1)
    if scale == 0.0:
        assert v[0, 0] == pytest.approx(1.0, abs=1e-9) and abs(v[0, 4]) < 1e-9   # no rolling either
    else:
        # friction brings it to rolling at 5/7 of its speed (a uniform sphere); the soft contact
        # leaves a slip of ~1e-3 m/s
        assert v[0, 0] == pytest.approx(5.0 / 7.0, abs=3e-3) and abs(v[0, 0] - 0.05 * v[0, 4]) < 3e-3


def _pd_arm(forcelimited=False):
    b = W.ModelBuilder("arm")
    link = b.body(0, (0, 0, 0))
    b.joint(link, W.HINGE, axis=(0, 0, 1))
    b.geom(link, W.CAPSULE, (0.02, 0.1), pos=(0.1, 0, 0), quat=(0.7071068, 0, 0.7071068, 0), mass=0.5)
    b.actuator(0, W.POSITION, kp=20.0, kd=1.0, forcelimited=forcelimited, forcerange=(-0.5, 0.8))
    return b.build(timestep=0.002, gravity=(0, 0, 0), iterations=4)


def test_calibration_offset_shifts_the_pd_equilibrium():
    m = _pd_arm()
    p = RZ.nominal(m); p[RZ.rows(m)["calibration"]] = 0.07
    om = O.OracleModel(RZ.substituted_model(m, p))
    u = RZ.controls(m, p, np.full((3000, 1, 1), 0.3))
    q, v, _, _ = om.rollout(np.zeros((1, 1)), np.zeros((1, 1)), u, 1)
    assert q[0, 0] == pytest.approx(0.37, abs=1e-6)


@pytest.mark.parametrize("err,expect", [(0.01, 0.2), (0.5, 0.8), (-0.5, -0.5)])
def test_torque_limits_clip_the_pd_force(err, expect):
    """tau = clip(kp (u - q) - kd qd, lo, hi) with kp 20, range (-0.5, 0.8)."""
    m = _pd_arm(forcelimited=True)
    f = O.OracleModel(m).forward(np.zeros(1), np.zeros(1), None, np.array([err]))
    assert f["actuator"][0] == pytest.approx(expect)


def test_pd_gain_scales_multiply_kp_and_kd():
    """tau = kp (1 + s_p) (u - q) - kd (1 + s_d) qd at a state with both terms non-zero (a swapped
    pair of rows or an additive reading fails)."""
    m = _pd_arm()
    R = RZ.rows(m)
    p = RZ.nominal(m); p[R["kp"]] = 0.3; p[R["kd"]] = -0.4
    q, qd, u = 0.1, 0.7, 0.35
    f = O.OracleModel(RZ.substituted_model(m, p)).forward(np.array([q]), np.array([qd]), None, np.array([u]))
    assert f["actuator"][0] == pytest.approx(20.0 * 1.3 * (u - q) - 1.0 * 0.6 * qd, rel=1e-12)


def test_link_mass_scale_scales_mass_and_inertia():
    """A single free body: every entry of its mass matrix scales by 1 + s (mass and the inertia
    about the centre of mass both), and resting on a plane the contacts carry (1 + s) m g."""
    m = _box_on_plane()
    R = RZ.rows(m)
    p = RZ.nominal(m); p[R["mass"] + 1] = 0.25
    q = np.array([0.1, -0.2, 0.3, np.cos(0.4), np.sin(0.4) * 0.6, 0.0, np.sin(0.4) * 0.8])
    M0 = O.OracleModel(m).mass_matrix(q)
    M1 = O.OracleModel(RZ.substituted_model(m, p)).mass_matrix(q)
    np.testing.assert_allclose(M1, 1.25 * M0, rtol=1e-12, atol=1e-15)
    om, qs, vs = _settle(m, p)
    assert _normal_force(om, qs, vs) == pytest.approx(1.25 * 2.0 * 9.81, rel=1e-6)


def test_link_mass_scale_comes_before_the_payload():
    """body 1's mass is (1 + s) m + payload: the payload is not scaled."""
    m = _box_on_plane()
    R = RZ.rows(m)
    p = RZ.nominal(m); p[R["mass"] + 1] = -0.5; p[1] = 1.0
    om, qs, vs = _settle(m, p)
    assert _normal_force(om, qs, vs) == pytest.approx((0.5 * 2.0 + 1.0) * 9.81, rel=1e-6)


def test_friction_loss_scale_sets_the_sliding_deceleration():
    """A spinning joint with friction loss F and scale s decelerates at F (1 + s) / I."""
    b = W.ModelBuilder("fric_arm")
    link = b.body(0, (0, 0, 0))
    b.joint(link, W.HINGE, axis=(0, 0, 1), frictionloss=0.3)
    b.geom(link, W.BOX, (0.2, 0.05, 0.05), pos=(0.2, 0, 0), mass=2.0)
    b.actuator(0, W.MOTOR, gear=1.0)
    m = b.build(timestep=0.002, gravity=(0, 0, 0), iterations=50)
    R = RZ.rows(m)
    p = RZ.nominal(m); p[R["frictionloss"]] = 0.6
    om = O.OracleModel(RZ.substituted_model(m, p))
    I = om.mass_matrix(np.zeros(1))[0, 0]
    f = om.forward(np.zeros(1), np.array([2.0]), None, np.array([0.0]), solver_cap=-1)
    assert f["qacc"][0] == pytest.approx(-float(np.float32(0.3)) * 1.6 / I, rel=1e-9)


def test_parameter_rows_partition_the_block():
    """the groups' first rows tile [0, nrand) in the documented order"""
    m = W.quadruped()
    R = RZ.rows(m)
    sizes = {"friction": 1, "payload": 1, "com": 3 * m.nbody, "armature": m.nv, "calibration": m.nu,
             "kp": m.nu, "kd": m.nu, "mass": m.nbody, "frictionloss": m.nv}
    at = 0
    for k in ("friction", "payload", "com", "armature", "calibration", "kp", "kd", "mass", "frictionloss"):
        assert R[k] == at
        at += sizes[k]
    assert at == RZ.nrand(m)
