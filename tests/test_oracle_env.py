"""Pins of the oracle's locomotion task layer (oracle/env.py) against closed forms, invariances
and finite differences, independent of the formulas it implements."""
import dataclasses
import math

import numpy as np
import pytest

from paper_2502_08844_b300 import workloads as W
from oracle import oracle as O
from oracle import env as E


@pytest.fixture(scope="module")
def quad():
    m = W.quadruped()
    om = O.OracleModel(m)
    return m, om, E.OracleTask(om, W.quadruped_task())


def _quat_axis(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * a])


def _qmul(a, b):
    w1, x1, y1, z1 = a; w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _rotz(psi):
    c, s = math.cos(psi), math.sin(psi)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])


def test_targets_absolute_and_relative(quad):
    m, om, ot = quad
    a1 = np.linspace(-1, 1, m.nu); a2 = np.cos(np.arange(m.nu))
    assert np.allclose(ot.targets(np.zeros(m.nu), None), ot.q_default)
    assert np.allclose(ot.targets(a1, None), ot.q_default + 0.3 * a1, atol=1e-7)
    rel = E.OracleTask(om, dataclasses.replace(W.quadruped_task(), action_mode=W.RELATIVE))
    q1 = rel.targets(a1, rel.q_default)
    q2 = rel.targets(a2, q1)
    assert np.allclose(q2, rel.q_default + 0.3 * (a1 + a2), atol=1e-7)   # relative targets accumulate


def test_targets_clip_to_a_limited_control_range():
    m = W.quadruped()
    m.act_ctrllimited[:] = 1
    m.act_ctrlrange[:] = np.array([-0.5, 0.5], np.float32)
    ot = E.OracleTask(O.OracleModel(m), W.quadruped_task())
    q = ot.targets(np.ones(m.nu), None)
    assert np.all(q <= 0.5 + 1e-12) and np.all(q >= -0.5 - 1e-12)
    assert q[0] == pytest.approx(0.3)              # abduction 0 + 0.3 stays inside
    assert q[1] == pytest.approx(0.5)              # flexion 0.9 + 0.3 is clipped at the top


def test_standing_observation(quad):
    m, om, ot = quad
    q = m.qpos_init.astype(np.float64); v = np.zeros(m.nv)
    cmd = np.array([0.4, -0.2, 0.7]); a = np.arange(m.nu) / 10.0
    o = ot.observation(q, v, a, cmd)
    assert o.shape == (12 + 3 * m.nu,)
    assert np.allclose(o[:3], [0, 0, -1])          # upright base: gravity straight down
    assert np.allclose(o[3:9 + 2 * m.nu], 0.0, atol=1e-12)   # at rest in the default pose
    assert np.allclose(o[9 + 2 * m.nu:9 + 3 * m.nu], a) and np.allclose(o[-3:], cmd)


@pytest.mark.parametrize("phi", [0.3, 1.2, 2.0, 3.0])
def test_rolled_base_gravity_and_termination(quad, phi):
    """Rolling the base by phi about x puts gravity at (0, -sin phi, -cos phi) in the base frame;
    the robot has turned over once cos phi < 0."""
    m, om, ot = quad
    q = m.qpos_init.astype(np.float64).copy(); q[2] += 0.5
    q[3:7] = _quat_axis((1, 0, 0), phi)
    o = ot.observation(q, np.zeros(m.nv), np.zeros(m.nu), np.zeros(3))
    assert np.allclose(o[:3], [0, -math.sin(phi), -math.cos(phi)], atol=1e-12)
    assert ot.terminated(q, np.zeros(m.nv)) == (math.cos(phi) < 0)
    v = np.zeros(m.nv); v[0] = np.nan
    assert ot.terminated(m.qpos_init.astype(np.float64), v)


def test_observation_and_reward_are_yaw_invariant(quad):
    """Turning the whole robot about the world z axis (its base orientation and its world
    linear velocity) changes nothing the task sees: every quantity is in the base frame."""
    m, om, ot = quad
    rng = np.random.default_rng(3)
    q = m.qpos_init.astype(np.float64).copy(); q[2] += 0.05
    q[3:7] = _quat_axis((0.3, -0.2, 1.0), 0.4)
    q[7:] += 0.1 * rng.standard_normal(m.nq - 7)
    v = 0.5 * rng.standard_normal(m.nv)
    q_des = ot.targets(rng.uniform(-1, 1, m.nu), None)
    a = rng.uniform(-1, 1, m.nu); ap = rng.uniform(-1, 1, m.nu); cmd = np.array([0.5, -0.3, 0.8])
    air = np.array([0.1, 0.0, 0.3, 0.05]); con = np.array([1.0, 0.0, 0.0, 1.0])
    o0 = ot.observation(q, v, ap, cmd)
    r0, air0, c0 = ot.terms(q, v, q_des, a, ap, cmd, air, con, 0.02, False)
    psi = 1.1
    q2 = q.copy(); q2[3:7] = _qmul(_quat_axis((0, 0, 1), psi), q[3:7]); q2[0:3] = _rotz(psi) @ q[0:3]
    v2 = v.copy(); v2[0:3] = _rotz(psi) @ v[0:3]
    o1 = ot.observation(q2, v2, ap, cmd)
    r1, air1, c1 = ot.terms(q2, v2, q_des, a, ap, cmd, air, con, 0.02, False)
    assert np.allclose(o0, o1, atol=1e-10)
    assert np.allclose(r0, r1, atol=1e-10) and np.allclose(air0, air1) and np.allclose(c0, c1)


def test_foot_velocity_matches_finite_differences(quad):
    m, om, ot = quad
    rng = np.random.default_rng(5)
    q = m.qpos_init.astype(np.float64).copy(); q[3:7] = _quat_axis((0.2, 1.0, 0.1), 0.3)
    q[7:] += 0.2 * rng.standard_normal(m.nq - 7)
    v = rng.standard_normal(m.nv)
    _, _, vel = ot.feet(q, v)
    eps = 1e-6
    pp, _, _ = ot.feet(om.integrate_pos(q, v, eps), v)
    pm, _, _ = ot.feet(om.integrate_pos(q, v, -eps), v)
    assert np.allclose(vel, (pp - pm) / (2 * eps), atol=1e-6)


def test_foot_heights_in_the_standing_pose(quad):
    """The standing pose puts every foot 1 mm above the plane; lifting the base lifts them."""
    m, om, ot = quad
    q = m.qpos_init.astype(np.float64).copy()
    _, h, _ = ot.feet(q, np.zeros(m.nv))
    assert np.allclose(h, 0.001, atol=2e-7)        # float32 model arrays
    q[2] += 0.03
    _, h2, _ = ot.feet(q, np.zeros(m.nv))
    assert np.allclose(h2 - h, 0.03, atol=1e-12)


def test_air_time_over_a_scripted_gait(quad):
    """Feet up for k control steps, then down: the touchdown step earns
    clip(k dt - T_min, 0, T_max - T_min) per foot, and nothing before or after."""
    m, om, ot = quad
    dt = 0.02
    up = m.qpos_init.astype(np.float64).copy(); up[2] += 0.05
    down = m.qpos_init.astype(np.float64).copy(); down[2] -= 0.0015   # below the 2 mm contact height
    v = np.zeros(m.nv); qd = ot.q_default; a = np.zeros(m.nu)
    for k, expect in [(3, 0.0), (10, 0.1), (40, 0.4)]:
        air, con = np.zeros(4), np.ones(4)
        for _ in range(k):
            r, air, con = ot.terms(up, v, qd, a, a, np.zeros(3), air, con, dt, False)
            assert r[E.T["air_time"]] == 0.0 and r[E.T["slip"]] == 0.0
        assert np.allclose(air, k * dt) and np.all(con == 0)
        r, air, con = ot.terms(down, v, qd, a, a, np.zeros(3), air, con, dt, False)
        per_foot = min(max((k + 1) * dt - 0.1, 0.0), 0.4)
        assert r[E.T["air_time"]] == pytest.approx(4 * per_foot) and np.all(air == 0) and np.all(con == 1)
        r, air, con = ot.terms(down, v, qd, a, a, np.zeros(3), air, con, dt, False)
        assert r[E.T["air_time"]] == 0.0       # still down: no second reward


def test_tracking_special_cases_and_clip(quad):
    m, om, ot = quad
    q = m.qpos_init.astype(np.float64).copy(); q[2] += 0.1
    v = np.zeros(m.nv); v[0], v[1], v[5] = 0.6, -0.2, 0.9      # base upright: base frame = world axes
    z = np.zeros(m.nu); con = np.zeros(4)
    r, _, _ = ot.terms(q, v, ot.q_default, z, z, np.array([0.6, -0.2, 0.9]), np.zeros(4), con, 0.02, False)
    assert r[E.T["lin_vel"]] == pytest.approx(1.0) and r[E.T["ang_vel"]] == pytest.approx(1.0)
    s = math.sqrt(0.25)
    r, _, _ = ot.terms(q, v, ot.q_default, z, z, np.array([0.6 + s, -0.2, 0.9 - s]), np.zeros(4), con, 0.02, False)
    assert r[E.T["lin_vel"]] == pytest.approx(math.exp(-1)) and r[E.T["ang_vel"]] == pytest.approx(math.exp(-1))
    assert r[E.T["stand_still"]] == pytest.approx(math.hypot(0.6 + s, -0.2))
    neg = E.OracleTask(om, W.quadruped_task(weights={k: -1.0 for k in W.TERMS}))
    assert neg.reward(r) == 0.0                    # a negative weighted sum is clipped to zero
    pos = E.OracleTask(om, W.quadruped_task(weights={k: (1.0 if k == "lin_vel" else 0.0) for k in W.TERMS}))
    assert pos.reward(r) == pytest.approx(math.exp(-1))


def test_pd_torque_and_energy(quad):
    """tau = kp (q_des - q) - kd qdot (eq. pd_mapping) on every actuated joint."""
    m, om, ot = quad
    q = m.qpos_init.astype(np.float64).copy(); q[2] += 0.1
    v = np.zeros(m.nv); v[6:] = 2.0
    q_des = ot.q_default + 0.1
    z = np.zeros(m.nu)
    r, _, _ = ot.terms(q, v, q_des, z, z, np.zeros(3), np.zeros(4), np.zeros(4), 0.02, False)
    tau = 35.0 * 0.1 - 0.5 * 2.0
    assert r[E.T["torque"]] == pytest.approx(m.nu * tau ** 2, rel=1e-6)
    assert r[E.T["energy"]] == pytest.approx(m.nu * abs(2.0 * tau), rel=1e-6)
    assert r[E.T["joint_pos"]] == pytest.approx(0.0) and r[E.T["pose"]] == pytest.approx(1.0)


def test_step_terminates_truncates_and_resets(quad):
    m, om, ot = quad
    q0 = m.qpos_init.astype(np.float64); v0 = np.zeros(m.nv)
    cmd = np.array([0.3, 0.0, 0.0]); a = np.full(m.nu, 0.2)
    # turned over: terminated, reset to (q0, v0), task state back to its defaults
    qf = q0.copy(); qf[2] += 0.3; qf[3:7] = _quat_axis((1, 0, 0), math.pi)
    st = ot.initial_task_state(); st[-1] = 5.0
    out = ot.step(qf, v0, np.zeros(m.nv), st, a, cmd, q0, v0, 5)
    assert out["terminated"] and out["done"] == 1.0 and out["truncated"] == 0.0
    assert out["terms"][E.T["termination"]] == 1.0
    assert np.array_equal(out["qpos"], q0) and np.array_equal(out["qvel"], v0) and np.all(out["warm"] == 0)
    assert np.array_equal(out["task_state"], ot.initial_task_state())
    assert np.allclose(out["obs"], ot.observation(q0, v0, np.zeros(m.nu), cmd))
    # upright, episode of one step: truncated (done, not terminated)
    short = E.OracleTask(om, W.quadruped_task(episode_length=1))
    out = short.step(q0, v0, np.zeros(m.nv), short.initial_task_state(), a, cmd, q0, v0, 5)
    assert out["done"] == 1.0 and out["truncated"] == 1.0 and out["terms"][E.T["termination"]] == 0.0
    # a running episode keeps the physics result and records the action
    out = ot.step(q0, v0, np.zeros(m.nv), ot.initial_task_state(), a, cmd, q0, v0, 5)
    assert out["done"] == 0.0 and np.array_equal(out["qpos"], out["qpos_final"])
    q_des, a_prev, air, con, step = ot.split(out["task_state"])
    assert np.allclose(q_des, ot.q_default + 0.3 * 0.2) and np.allclose(a_prev, a) and step == 1.0
    assert np.allclose(out["obs"][9 + 2 * m.nu:9 + 3 * m.nu], a)


def test_remaining_terms_in_closed_form(quad):
    """A base translating at (u, 0, vz) and spinning at (wx, wy, 0), rolled by phi, over feet at
    known heights: every foot moves with the base, so the clearance and slip terms follow from
    the heights and u alone."""
    m, om, ot = quad
    phi, u, vz, wx, wy = 0.2, 0.7, 0.4, 0.3, -0.4
    q = m.qpos_init.astype(np.float64).copy()
    q[3:7] = _quat_axis((1, 0, 0), phi)
    _, h, _ = ot.feet(q, np.zeros(m.nv))
    v = np.zeros(m.nv); v[0], v[2] = u, vz
    a = np.linspace(-1, 1, m.nu); ap = a[::-1].copy()
    r, _, _ = ot.terms(q, v, ot.q_default, a, ap, np.zeros(3), np.zeros(4), np.zeros(4), 0.02, False)
    assert r[E.T["orientation"]] == pytest.approx(math.sin(phi) ** 2)
    # base-frame vertical speed of a world velocity (u, 0, vz) under a roll about x
    assert r[E.T["lin_z"]] == pytest.approx((vz * math.cos(phi)) ** 2)
    assert r[E.T["action_rate"]] == pytest.approx(np.sum((a - ap) ** 2))
    assert r[E.T["clearance"]] == pytest.approx(np.sum((h - 0.08) ** 2) * math.sqrt(u))
    assert r[E.T["slip"]] == pytest.approx(np.sum(h < 0.002) * u * u)
    v = np.zeros(m.nv); v[3], v[4] = wx, wy
    r, _, _ = ot.terms(q, v, ot.q_default, a, a, np.zeros(3), np.zeros(4), np.zeros(4), 0.02, False)
    assert r[E.T["ang_xy"]] == pytest.approx(wx * wx + wy * wy) and r[E.T["action_rate"]] == 0.0
