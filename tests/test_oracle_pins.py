"""Pins of the FP64 oracle against things other than itself: values the paper prints, closed
forms, invariants, special cases that reduce to textbook results, and brute force on tiny
inputs.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_08844_b300 import workloads as W
from tests import models_for_tests as TM

HERE = os.path.dirname(os.path.abspath(__file__))
G = 9.81


def rng(seed):
    return np.random.default_rng(seed)


def random_quat(r):
    q = r.normal(size=4)
    return q / np.linalg.norm(q)


def quat_to_mat(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def random_rot(r):
    # a random orthonormal matrix from a QR decomposition (independent of the quaternion formula)
    Q, R = np.linalg.qr(r.normal(size=(3, 3)))
    Q = Q @ np.diag(np.sign(np.diag(R)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


# --------------------------------------------------------------------------------------
# model compiler: armature and solid inertias
# --------------------------------------------------------------------------------------

def test_armature_matches_paper_worked_example():
    g = json.load(open(os.path.join(HERE, "golden", "armature_leap.json")))
    Ir = 0.5 * g["m_r"] * g["r_r"] ** 2
    # the paper rounds the rotor inertia to 1.7e-8
    assert abs(Ir - g["I_r_printed"]) <= g["I_r_printed_rounding"]
    Ia = O.rotor_armature(g["k_g"], g["m_r"], g["r_r"])
    assert Ia == pytest.approx(g["k_g"] ** 2 * Ir, rel=1e-14)
    assert Ia == pytest.approx(g["k_g"] ** 2 * g["I_r_printed"], rel=0.02)
    assert Ia == pytest.approx(1.4135e-3, rel=0.02)


def _grid_inertia(inside, lo, hi, n):
    """Inertia tensor diagonal (about the origin) of a uniform unit-mass solid by midpoint grid integration."""
    axes = [np.linspace(lo[k], hi[k], n, endpoint=False) + (hi[k] - lo[k]) / (2 * n) for k in range(3)]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    mask = inside(X, Y, Z)
    cnt = mask.sum()
    Ixx = ((Y ** 2 + Z ** 2) * mask).sum() / cnt
    Iyy = ((X ** 2 + Z ** 2) * mask).sum() / cnt
    Izz = ((X ** 2 + Y ** 2) * mask).sum() / cnt
    return np.array([Ixx, Iyy, Izz])


@pytest.mark.parametrize("gtype,size", [(W.SPHERE, (0.1,)), (W.BOX, (0.19, 0.05, 0.05)),
                                        (W.CAPSULE, (0.02, 0.1)), (W.CAPSULE, (0.05, 0.5))])
def test_solid_inertia_matches_grid_integration(gtype, size):
    m = 1.7
    if gtype == W.SPHERE:
        r = size[0]
        ins = lambda X, Y, Z: X ** 2 + Y ** 2 + Z ** 2 <= r * r
        lo, hi = [-r] * 3, [r] * 3
    elif gtype == W.BOX:
        h = size
        ins = lambda X, Y, Z: (np.abs(X) <= h[0]) & (np.abs(Y) <= h[1]) & (np.abs(Z) <= h[2])
        lo, hi = [-x for x in h], list(h)
    else:
        r, hl = size
        ins = lambda X, Y, Z: X ** 2 + Y ** 2 + (np.maximum(np.abs(Z) - hl, 0.0)) ** 2 <= r * r
        lo, hi = [-r, -r, -hl - r], [r, r, hl + r]
    I = m * _grid_inertia(ins, lo, hi, 240)
    assert np.allclose(O.solid_inertia(gtype, size, m), I, rtol=1e-2)


# --------------------------------------------------------------------------------------
# kinematics
# --------------------------------------------------------------------------------------

def test_fk_planar_chain_closed_form():
    L = 0.5
    om = O.OracleModel(TM.planar_chain(3, length=L))
    r = rng(1)
    for _ in range(5):
        q = r.uniform(-3, 3, size=3)
        R, x, com = om.body_frames(q)
        p = np.zeros(3)
        phi = 0.0
        for i in range(3):
            phi += q[i]
            d = np.array([-L * math.sin(phi), 0.0, -L * math.cos(phi)])
            assert np.allclose(x[i + 1], p, atol=1e-12)
            assert np.allclose(com[i + 1], p + d / 2, atol=1e-12)
            Ry = np.array([[math.cos(phi), 0, math.sin(phi)], [0, 1, 0], [-math.sin(phi), 0, math.cos(phi)]])
            assert np.allclose(R[i + 1], Ry, atol=1e-12)
            p = p + d


def test_fk_hinge_full_turn_is_identity_and_rotations_orthonormal():
    om = O.OracleModel(W.quadruped())
    q0 = W.quadruped().qpos_init.astype(np.float64)
    q1 = q0.copy()
    q1[7:] += 2 * math.pi
    R0, x0, _ = om.body_frames(q0)
    R1, x1, _ = om.body_frames(q1)
    assert np.allclose(R0, R1, atol=1e-12) and np.allclose(x0, x1, atol=1e-12)
    r = rng(2)
    q = q0.copy()
    q[3:7] = random_quat(r) * 3.0   # unnormalised input quaternion is normalised by FK
    q[7:] = r.uniform(-2, 2, 12)
    R, _, _ = om.body_frames(q)
    for Rb in R:
        assert np.allclose(Rb @ Rb.T, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(Rb) - 1) < 1e-12
    assert np.allclose(R[1], quat_to_mat(q[3:7] / np.linalg.norm(q[3:7])), atol=1e-12)


def test_fk_cartpole_closed_form():
    om = O.OracleModel(W.cartpole())
    for x, th in [(0.3, 0.2), (-1.0, 2.5)]:
        R, xb, com = om.body_frames([x, th])
        assert np.allclose(com[1], [x, 0, 0], atol=1e-12)
        assert np.allclose(com[2], [x + 0.5 * math.sin(th), 0, 0.5 * math.cos(th)], atol=1e-12)


# --------------------------------------------------------------------------------------
# mass matrix and bias forces
# --------------------------------------------------------------------------------------

def _random_quadruped_state(r):
    m = W.quadruped()
    q = m.qpos_init.astype(np.float64).copy()
    q[:3] = r.uniform(-1, 1, 3)
    q[3:7] = random_quat(r)
    q[7:] += r.uniform(-0.5, 0.5, 12)
    v = r.uniform(-2, 2, 18)
    return m, q, v


def test_mass_matrix_equals_inverse_dynamics_columns_and_is_spd():
    r = rng(3)
    m, q, v = _random_quadruped_state(r)
    om = O.OracleModel(m)
    M = om.mass_matrix(q)
    nv = om.nv
    base = om.inverse_dynamics(q, np.zeros(nv), np.zeros(nv))
    cols = np.stack([om.inverse_dynamics(q, np.zeros(nv), np.eye(nv)[j]) - base for j in range(nv)], axis=1)
    assert np.allclose(M, cols, rtol=1e-12, atol=1e-12)
    assert np.allclose(M, M.T, atol=1e-13)
    assert np.linalg.eigvalsh(M).min() > 0
    # kinetic energy from per-body velocities
    T, _ = om.energy(q, v)
    assert 0.5 * v @ M @ v == pytest.approx(T, rel=1e-12)


def test_cartpole_mass_matrix_and_gravity_closed_form():
    om = O.OracleModel(W.cartpole())
    mc, mp, l = 1.0, 0.1, 0.5
    Ip = O.solid_inertia(W.CAPSULE, (0.05, 0.5), mp)[0]
    for th in [0.0, 0.7, -2.0]:
        M = om.mass_matrix([0.2, th])
        Mref = np.array([[mc + mp, mp * l * math.cos(th)], [mp * l * math.cos(th), mp * l * l + Ip]])
        assert np.allclose(M, Mref, rtol=1e-6)   # float32-rounded model values
        c = om.inverse_dynamics([0.2, th], [0, 0], [0, 0])
        assert np.allclose(c, [0, -mp * G * l * math.sin(th)], rtol=1e-6, atol=1e-9)


def test_gravity_forces_are_potential_gradient():
    """c(q, 0) = dU/dq, with the directional derivative taken along each dof by the integrator."""
    r = rng(4)
    m, q, _ = _random_quadruped_state(r)
    om = O.OracleModel(m)
    c = om.inverse_dynamics(q, np.zeros(om.nv), np.zeros(om.nv))
    eps = 1e-6
    grad = np.zeros(om.nv)
    for k in range(om.nv):
        e = np.eye(om.nv)[k]
        Up = om.energy(om.integrate_pos(q, e, eps), np.zeros(om.nv))[1]
        Um = om.energy(om.integrate_pos(q, e, -eps), np.zeros(om.nv))[1]
        grad[k] = (Up - Um) / (2 * eps)
    assert np.allclose(c, grad, rtol=1e-6, atol=1e-7)


def test_velocity_terms_match_lagrangian_fixed_base():
    """c(q,qd) - g(q) = Mdot qd - 1/2 d/dq (qd^T M qd) for true generalised coordinates (hinges)."""
    m = TM.planar_chain(3, length=0.4, gravity=(0, 0, 0))
    om = O.OracleModel(m)
    r = rng(5)
    q, v = r.uniform(-2, 2, 3), r.uniform(-3, 3, 3)
    c = om.inverse_dynamics(q, v, np.zeros(3))
    eps = 1e-6
    Mdot = (om.mass_matrix(q + eps * v) - om.mass_matrix(q - eps * v)) / (2 * eps)
    dKE = np.array([(v @ om.mass_matrix(q + eps * e) @ v - v @ om.mass_matrix(q - eps * e) @ v) / (2 * eps)
                    for e in np.eye(3)])
    assert np.allclose(c, Mdot @ v - 0.5 * dKE, rtol=1e-6, atol=1e-8)


def test_velocity_terms_match_lagrangian_slider_on_rotating_arm():
    m = TM.arm_with_slider()
    om = O.OracleModel(m)
    r = rng(15)
    for _ in range(3):
        q, v = r.uniform(-1, 1, 3), r.uniform(-3, 3, 3)
        c = om.inverse_dynamics(q, v, np.zeros(3))
        eps = 1e-6
        Mdot = (om.mass_matrix(q + eps * v) - om.mass_matrix(q - eps * v)) / (2 * eps)
        dKE = np.array([(v @ om.mass_matrix(q + eps * e) @ v - v @ om.mass_matrix(q - eps * e) @ v) / (2 * eps)
                        for e in np.eye(3)])
        assert np.allclose(c, Mdot @ v - 0.5 * dKE, rtol=1e-6, atol=1e-8)


def test_energy_drift_floating_base_scales_with_timestep():
    drifts = []
    for h in (1e-3, 5e-4):
        m = TM.quadruped_passive(timestep=h)
        om = O.OracleModel(m)
        n = int(0.5 / h)
        q = m.qpos_init.astype(np.float64)[None].copy()
        v = rng(16).uniform(-2, 2, (1, 18))
        _, _, _, _, tq, tv = om.rollout(q, v, np.zeros((n, 1, 12)), 1, trajectory=True)
        E0 = sum(om.energy(q[0], v[0]))
        E = np.array([sum(om.energy(tq[i, 0], tv[i, 0])) for i in range(0, n, 5)])
        drifts.append(np.max(np.abs(E - E0)) / abs(E0))
    assert drifts[0] < 2e-2
    assert 1.5 < drifts[0] / drifts[1] < 2.8


def test_free_body_euler_equations():
    """One free body, COM at the origin, zero gravity: c = (0, w x I w) in body coordinates."""
    I6 = (0.3, 0.5, 0.7, 0.05, -0.02, 0.04)
    om = O.OracleModel(TM.free_body(gravity=(0, 0, 0), inertia=I6))
    r = rng(6)
    q = np.concatenate([r.normal(size=3), random_quat(r)])
    v = r.normal(size=6)
    c = om.inverse_dynamics(q, v, np.zeros(6))
    Il = np.array([[I6[0], I6[3], I6[4]], [I6[3], I6[1], I6[5]], [I6[4], I6[5], I6[2]]])
    Il = Il.astype(np.float32).astype(np.float64)
    w = v[3:]
    assert np.allclose(c[:3], 0, atol=1e-12)
    assert np.allclose(c[3:], np.cross(w, Il @ w), rtol=1e-7, atol=1e-9)


# --------------------------------------------------------------------------------------
# integrator and whole-step invariants
# --------------------------------------------------------------------------------------

def test_free_fall_is_exact_discrete():
    h, n = 0.01, 50
    m = TM.free_body(timestep=h, z0=10.0)
    om = O.OracleModel(m)
    q = np.array([0, 0, 10.0, 1, 0, 0, 0]); v = np.zeros(6)
    q2, v2, _, st = om.rollout(q[None], v[None], np.zeros((n, 1, 0)), 1)
    g = float(np.float32(9.81))
    h = float(np.float32(h))   # the model stores float32-rounded values
    assert st[0] == 0
    assert v2[0, 2] == pytest.approx(-g * n * h, rel=1e-12)
    assert q2[0, 2] == pytest.approx(10.0 - g * h * h * n * (n + 1) / 2, rel=1e-12)


def _period(om, theta0, h, T_total):
    n = int(T_total / h)
    q = np.array([[theta0]]); v = np.array([[0.0]])
    _, _, _, _, tq, _ = om.rollout(q, v, np.zeros((n, 1, 0)), 1, trajectory=True)
    th = np.concatenate([[theta0], tq[:, 0, 0]])
    t = np.arange(n + 1) * h
    # downward zero crossings (theta goes + -> -)
    idx = np.where((th[:-1] > 0) & (th[1:] <= 0))[0]
    tc = t[idx] + h * th[idx] / (th[idx] - th[idx + 1])
    return np.mean(np.diff(tc))


def test_pendulum_small_angle_period_and_convergence():
    theta0 = 0.05
    errs = []
    for h in (2e-3, 1e-3, 5e-4):
        m = TM.pendulum(timestep=h)
        om = O.OracleModel(m)
        mass, _, inertia, _ = om.massprops()
        lc = 0.5
        Ipiv = inertia[1, 1] + mass[1] * lc ** 2
        g = float(np.float32(9.81))
        T0 = 2 * math.pi * math.sqrt(Ipiv / (mass[1] * g * lc))
        Tex = T0 * (1 + theta0 ** 2 / 16 + 11 * theta0 ** 4 / 3072)
        errs.append(abs(_period(om, theta0, h, 12.0) - Tex) / Tex)
    assert errs[0] < 1e-4
    assert errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1]


def _energy_drift(h, T=2.0):
    m = TM.planar_chain(3, length=0.4, timestep=h)
    om = O.OracleModel(m)
    n = int(T / h)
    q = np.array([[1.0, -0.5, 0.8]]); v = np.array([[0.0, 1.0, -1.0]])
    _, _, _, _, tq, tv = om.rollout(q, v, np.zeros((n, 1, 0)), 1, trajectory=True)
    E0 = sum(om.energy(q[0], v[0]))
    E = np.array([sum(om.energy(tq[i, 0], tv[i, 0])) for i in range(0, n, 10)])
    return np.max(np.abs(E - E0)) / abs(E0)


def test_energy_drift_scales_with_timestep():
    d1, d2 = _energy_drift(1e-3), _energy_drift(5e-4)
    assert d1 < 2e-2
    assert 1.5 < d1 / d2 < 2.8


def _momentum_drift(h, T=0.4):
    m = TM.quadruped_zero_gravity(timestep=h)
    om = O.OracleModel(m)
    n = int(T / h)
    q0, v0 = W.initial_state(m, 1, 1)
    v0 = v0.astype(np.float64)
    ctrl = np.repeat(W.actions(m, 1, 1, 0, 1), n, axis=0)
    _, _, _, _, tq, tv = om.rollout(q0, v0, ctrl, 1, trajectory=True)
    P0, L0, _ = om.momentum(q0[0], v0[0])
    dP = max(np.linalg.norm(om.momentum(tq[i, 0], tv[i, 0])[0] - P0) for i in range(n))
    dL = max(np.linalg.norm(om.momentum(tq[i, 0], tv[i, 0])[1] - L0) for i in range(n))
    return dP, dL


def test_momentum_conservation_zero_gravity():
    dP1, dL1 = _momentum_drift(2e-3)
    dP2, dL2 = _momentum_drift(1e-3)
    # first-order drift (semi-implicit Euler evaluates M at the old configuration)
    assert dP1 < 0.1 and dL1 < 0.01
    assert 0.4 < dP2 / dP1 < 0.6 and 0.4 < dL2 / dL1 < 0.6


def test_free_body_linear_momentum_exact():
    om = O.OracleModel(TM.free_body(gravity=(0, 0, 0), inertia=(0.3, 0.5, 0.7, 0.05, -0.02, 0.04)))
    q = np.array([[0, 0, 1.0, 1, 0, 0, 0]]); v = np.array([[0.3, -0.2, 0.1, 2.0, -1.0, 3.0]])
    q2, v2, _, _ = om.rollout(q, v, np.zeros((300, 1, 0)), 1)
    assert np.array_equal(v2[0, :3], v[0, :3])


# --------------------------------------------------------------------------------------
# soft contact model and solver
# --------------------------------------------------------------------------------------

def test_impedance_closed_form_points():
    si = [0.9, 0.95, 0.001, 0.5, 2.0]
    assert O.impedance(0.0, si) == pytest.approx(0.9)
    assert O.impedance(-0.001, si) == pytest.approx(0.95)
    assert O.impedance(-0.5, si) == pytest.approx(0.95)
    assert O.impedance(-0.0005, si) == pytest.approx(0.925)      # x = mid: y = mid
    assert O.impedance(-0.00025, si) == pytest.approx(0.9 + 0.05 * 0.125)   # y = x^2/mid
    assert O.impedance(-0.00075, si) == pytest.approx(0.9 + 0.05 * (1 - 0.125))
    for r in (-0.0005 + 1e-12, -0.0005 - 1e-12):   # continuity at mid
        assert abs(O.impedance(r, si) - 0.925) < 1e-9


def test_sphere_rests_on_plane_at_predicted_penetration():
    m = TM.sphere_on_plane(mass=1.0, radius=0.1, friction=0.0, condim=1, timestep=0.002)
    om = O.OracleModel(m)
    q = np.array([[0, 0, 0.1, 1, 0, 0, 0]]); v = np.zeros((1, 6))
    q2, v2, _, st = om.rollout(q, v, np.zeros((1000, 1, 0)), 1)
    assert np.linalg.norm(v2) < 1e-6
    # steady state: m g = D(r) k d(r) (-r), D = d / ((1-d) Ahat), Ahat = 1/m
    si = [float(np.float32(x)) for x in (0.9, 0.95, 0.001, 0.5, 2.0)]
    tc, dmax = float(np.float32(0.02)), si[1]
    k = 1.0 / (dmax * dmax * tc * tc)
    g = float(np.float32(9.81))

    def resid(r):
        d = O.impedance(r, si)
        return d / ((1 - d) * 1.0) * k * d * (-r) - g

    lo, hi = -0.01, -1e-12
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if resid(mid) > 0:
            lo = mid
        else:
            hi = mid
    r_star = 0.5 * (lo + hi)
    radius = float(np.float32(0.1))
    assert (q2[0, 2] - radius) == pytest.approx(r_star, rel=1e-6)


def test_sphere_with_friction_comes_to_rest():
    m = TM.sphere_on_plane(mass=1.0, radius=0.1, friction=1.0, condim=3, timestep=0.002)
    om = O.OracleModel(m)
    q = np.array([[0, 0, 0.101, 1, 0, 0, 0]]); v = np.zeros((1, 6))
    q2, v2, _, _ = om.rollout(q, v, np.zeros((1000, 1, 0)), 1)
    assert np.linalg.norm(v2) < 1e-6


def test_sliding_sphere_ends_rolling_at_five_sevenths():
    """A solid sphere launched sliding (v0, no spin) on a plane with friction ends rolling without
    slip at 5/7 v0: angular momentum about the contact line is conserved."""
    m = TM.sphere_on_plane(mass=1.0, radius=0.1, friction=1.0, condim=3, timestep=0.002)
    om = O.OracleModel(m)
    v0 = 0.05
    q = np.array([[0, 0, 0.1, 1, 0, 0, 0]]); v = np.array([[v0, 0.0, 0, 0, 0, 0]])
    q2, v2, _, _ = om.rollout(q, v, np.zeros((1000, 1, 0)), 1)
    assert v2[0, 0] == pytest.approx(5.0 / 7.0 * v0, rel=3e-3)
    assert v2[0, 4] * 0.1 == pytest.approx(v2[0, 0], rel=3e-3)   # no slip: v = w r


def _random_problem(r, nv, nr):
    A = r.normal(size=(nv, nv))
    M = A @ A.T + nv * np.eye(nv)
    J = r.normal(size=(nr, nv))
    a0 = r.normal(size=nv)
    aref = r.normal(size=nr) * 3
    D = r.uniform(0.5, 5.0, size=nr)
    return M, a0, J, aref, D


def _brute_force(M, a0, J, aref, D):
    nr = J.shape[0]
    sols = []
    for mask in range(1 << nr):
        S = np.array([(mask >> i) & 1 for i in range(nr)], bool)
        H = M + (J[S].T * D[S]) @ J[S]
        a = np.linalg.solve(H, M @ a0 + (J[S].T * D[S]) @ aref[S])
        if np.array_equal((J @ a - aref) < 0, S):
            sols.append(a)
    return sols


@pytest.mark.parametrize("seed", range(12))
def test_newton_converged_equals_brute_force_active_set(seed):
    r = rng(100 + seed)
    nv, nr = 6, [2, 5, 8][seed % 3]
    M, a0, J, aref, D = _random_problem(r, nv, nr)
    sols = _brute_force(M, a0, J, aref, D)
    assert len(sols) == 1
    qacc, force, it, conv = O.solve(M, a0, J, aref, D, cap=-1)
    assert conv
    assert np.allclose(qacc, sols[0], rtol=1e-10, atol=1e-10)
    jar = J @ qacc - aref
    assert np.allclose(force, np.where(jar < 0, -D * jar, 0.0), rtol=1e-12, atol=1e-12)
    # optimality: M (a - a0) = J^T f
    assert np.allclose(M @ (qacc - a0), J.T @ force, rtol=1e-9, atol=1e-9)


def test_newton_capped_decreases_cost_and_respects_cap():
    r = rng(7)
    M, a0, J, aref, D = _random_problem(r, 8, 8)
    f_prev = O.cost(M, a0, J, aref, D, a0)
    for cap in (1, 2, 3):
        qacc, _, it, _ = O.solve(M, a0, J, aref, D, cap=cap)
        assert it <= cap
        f = O.cost(M, a0, J, aref, D, qacc)
        assert f <= f_prev + 1e-12
        f_prev = f


def test_quadruped_standing_forces_balance_weight():
    m = W.quadruped()
    om = O.OracleModel(m)
    q, v = W.initial_state(m, 1, 1)
    u = np.tile(m.default_ctrl[None, None, :], (200, 1, 1))
    q2, v2, w, st = om.rollout(q, v, u, 5)
    f = om.forward(q2[0], v2[0], w[0], u[0, 0], solver_cap=-1)
    mass = om.massprops()[0].sum()
    assert f["rows"][:, -1].sum() == pytest.approx(mass * float(np.float32(9.81)), rel=1e-3)


# --------------------------------------------------------------------------------------
# collision (model-free) against brute force
# --------------------------------------------------------------------------------------

def _sphere_points(n=200):
    th = np.linspace(0, math.pi, n)
    ph = np.linspace(0, 2 * math.pi, 2 * n)
    T, P = np.meshgrid(th, ph, indexing="ij")
    return np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)


def test_sphere_plane_brute_force():
    r = rng(8)
    for _ in range(5):
        R1 = random_rot(r); p1 = r.normal(size=3)
        c = r.normal(size=3); rad = 0.3
        out = O.collide(W.PLANE, R1, p1, [0, 0, 0], W.SPHERE, np.eye(3), c, [rad])
        n = R1[:, 2]
        pts = c + rad * _sphere_points()
        h = (pts - p1) @ n
        assert out[0, 0] == pytest.approx(h.min(), abs=1e-4)
        assert np.allclose(out[0, 4:7], n)


def _box_surface(h, n=60):
    g = np.linspace(-1, 1, n)
    A, B = np.meshgrid(g, g, indexing="ij")
    A, B = A.ravel(), B.ravel()
    faces = []
    for k in range(3):
        u, v = (k + 1) % 3, (k + 2) % 3
        for s in (-1, 1):
            P = np.zeros((A.size, 3))
            P[:, k] = s * h[k]; P[:, u] = A * h[u]; P[:, v] = B * h[v]
            faces.append(P)
    return np.concatenate(faces)


def test_sphere_box_brute_force():
    r = rng(9)
    h = np.array([0.2, 0.1, 0.15])
    for trial in range(8):
        R2 = random_rot(r); p2 = r.normal(size=3) * 0.1
        local = r.uniform(-1.5, 1.5, 3) * h if trial % 2 == 0 else r.uniform(-0.8, 0.8, 3) * h
        c = p2 + R2 @ local
        rad = 0.05
        out = O.collide(W.SPHERE, np.eye(3), c, [rad], W.BOX, R2, p2, h)
        surf = p2 + _box_surface(h, 120) @ R2.T
        dmin = np.linalg.norm(surf - c, axis=1).min()
        inside = np.all(np.abs(local) <= h)
        expected = (-dmin if inside else dmin) - rad
        assert out[0, 0] == pytest.approx(expected, abs=2e-3 * h.max())


def test_capsule_capsule_brute_force():
    r = rng(10)
    for _ in range(8):
        R1, R2 = random_rot(r), random_rot(r)
        p1, p2 = r.normal(size=3) * 0.2, r.normal(size=3) * 0.2
        s1, s2 = [0.05, 0.3], [0.04, 0.2]
        out = O.collide(W.CAPSULE, R1, p1, s1, W.CAPSULE, R2, p2, s2)
        lo1, hi1, lo2, hi2 = -s1[1], s1[1], -s2[1], s2[1]
        for _ in range(6):   # grid search, then refine around the best grid point
            u = np.linspace(lo1, hi1, 401); v = np.linspace(lo2, hi2, 401)
            P = p1 + u[:, None] * R1[:, 2]; Q = p2 + v[:, None] * R2[:, 2]
            D = np.linalg.norm(P[:, None, :] - Q[None, :, :], axis=-1)
            i, j = np.unravel_index(np.argmin(D), D.shape)
            du, dv = 3 * (hi1 - lo1) / 400, 3 * (hi2 - lo2) / 400
            lo1, hi1 = max(-s1[1], u[i] - du), min(s1[1], u[i] + du)
            lo2, hi2 = max(-s2[1], v[j] - dv), min(s2[1], v[j] + dv)
        d = D.min() - s1[0] - s2[0]
        assert out[0, 0] == pytest.approx(d, abs=1e-9)


def test_box_plane_deepest_corners():
    r = rng(11)
    h = np.array([0.1, 0.04, 0.015])
    for _ in range(5):
        R2 = random_rot(r); p2 = np.array([0, 0, 0.05]) + r.normal(size=3) * 0.01
        out = O.collide(W.PLANE, np.eye(3), np.zeros(3), [0, 0, 0], W.BOX, R2, p2, h)
        surf = p2 + _box_surface(h, 40) @ R2.T
        assert out[:, 0].min() == pytest.approx(surf[:, 2].min(), abs=1e-12)
        # the four reported depths are the four smallest corner heights
        corners = np.array([[sx, sy, sz] for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)]) * h
        zc = np.sort((p2 + corners @ R2.T)[:, 2])[:4]
        assert np.allclose(np.sort(out[:, 0]), zc, atol=1e-12)


def _support(R, p, h, u):
    return u @ p + np.abs(u @ R) @ h


def _sampled_depth(dirs, RA, pA, hA, RB, pB, hB, refine=True):
    """Penetration depth = min over unit directions u of s_A(u) + s_B(-u) (support functions):
    the minimum over the sampled directions, then a shrinking random local search around it
    (the minimum can sit on a cusp at an edge-edge direction)."""
    f = lambda D: D @ pA + np.abs(D @ RA) @ hA - (D @ pB) + np.abs(D @ RB) @ hB
    vals = f(dirs)
    best = dirs[np.argmin(vals)]
    fb = vals.min()
    if refine:
        gen = np.random.default_rng(0)
        step = 0.05
        for _ in range(60):
            cand = best + step * gen.normal(size=(2000, 3))
            cand /= np.linalg.norm(cand, axis=1, keepdims=True)
            fc = f(cand)
            if fc.min() < fb:
                fb, best = fc.min(), cand[np.argmin(fc)]
            step *= 0.8
    return fb


def test_box_box_depth_matches_sampled_support_overlap():
    r = rng(12)
    hA = np.array([0.06, 0.05, 0.01]); hB = np.array([0.035, 0.035, 0.035])
    dirs = r.normal(size=(200000, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    for trial in range(24):
        RA, RB = random_rot(r), random_rot(r)
        pA = np.zeros(3)
        u = r.normal(size=3); u /= np.linalg.norm(u)
        target = 0.002 if trial % 2 == 0 else 0.03   # shallow / deep overlap
        lo, hi = 0.0, 0.3                            # place B along u at that sampled depth
        for _ in range(50):
            t = 0.5 * (lo + hi)
            if _sampled_depth(dirs, RA, pA, hA, RB, t * u, hB, refine=False) > target:
                lo = t
            else:
                hi = t
        pB = 0.5 * (lo + hi) * u
        depth = _sampled_depth(dirs, RA, pA, hA, RB, pB, hB)
        out = O.collide(W.BOX, RA, pA, hA, W.BOX, RB, pB, hB)
        got = -out[:, 0].min()
        assert got <= depth + 1e-9             # no contact deeper than the penetration depth
        if target < 0.01:                      # shallow: the deepest contact is the penetration depth
            assert got == pytest.approx(depth, abs=1e-7)
        else:
            assert got > 0


def test_box_resting_on_box_gives_four_corner_contacts():
    hA = [0.06, 0.05, 0.01]; hB = [0.035, 0.035, 0.035]
    pA = np.zeros(3); pB = np.array([0.005, -0.004, 0.01 + 0.035 - 0.001])
    out = O.collide(W.BOX, np.eye(3), pA, hA, W.BOX, np.eye(3), pB, hB)
    assert np.allclose(out[:, 0], -0.001, atol=1e-12)
    assert np.allclose(out[:, 4:7], [0, 0, 1])
    xs = sorted(map(tuple, np.round(out[:, 1:3], 9)))
    exp = sorted((pB[0] + sx * 0.035, pB[1] + sy * 0.035) for sx in (-1, 1) for sy in (-1, 1))
    assert np.allclose(xs, exp, atol=1e-9)
    assert np.allclose(out[:, 3], 0.01 - 0.0005, atol=1e-12)
