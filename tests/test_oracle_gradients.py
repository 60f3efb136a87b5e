"""Pins of the oracle's reverse-mode rollout gradient against FP64 central differences
(step 1e-6) with the converged solver.  CPU only."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_08844_b300 import workloads as W

EPS = 1e-6


def _setup(T=4, env=0):
    m = W.quadruped()
    om = O.OracleModel(m)
    q0, v0 = W.initial_state(m, 4, env + 1)
    U = W.actions(m, 4, env + 1, 0, T)[:, env]
    w = O.tracking_loss_weights(om)
    mass, _, _, _ = om.massprops()
    return m, om, q0[env].astype(np.float64), v0[env].astype(np.float64), U.astype(np.float64), w, mass


def _fd(f, x, idx):
    out = []
    for i in idx:
        xp, xm = x.copy(), x.copy()
        xp.flat[i] += EPS
        xm.flat[i] -= EPS
        out.append((f(xp) - f(xm)) / (2 * EPS))
    return np.array(out)


def _close(a, b, rtol=1e-4, atol=1e-6):
    a, b = np.asarray(a), np.asarray(b)
    scale = max(np.abs(b).max(), 1e-12)
    assert np.abs(a - b).max() <= rtol * scale + atol, (a, b)


def test_gradient_matches_central_differences_state_and_controls():
    m, om, q0, v0, U, w, mass = _setup()
    g = O.rollout_grad(om, q0, v0, U, 5, w)
    assert g["loss"] == pytest.approx(O.rollout_loss(om, q0, v0, U, 5, w), rel=1e-12)
    # qpos: torso position, a quaternion component and the leg joints; qvel all
    qi = [0, 1, 2, 4, 7, 9, 12, 15, 18]
    _close(g["q0"][qi], _fd(lambda x: O.rollout_loss(om, x, v0, U, 5, w), q0, qi))
    vi = list(range(18))
    _close(g["v0"][vi], _fd(lambda x: O.rollout_loss(om, q0, x, U, 5, w), v0, vi))
    ui = [0, 5, 11, 12 + 3, 36 + 8]
    _close(g["u"].flat[ui], _fd(lambda x: O.rollout_loss(om, q0, v0, x.reshape(U.shape), 5, w), U, ui))


def test_gradient_matches_central_differences_parameters():
    m, om, q0, v0, U, w, mass = _setup()
    damping = np.zeros(18)
    kp = np.full(12, float(np.float32(35.0)))
    g = O.rollout_grad(om, q0, v0, U, 5, w, mass=mass, damping=damping, kp=kp)
    bi = list(range(1, 10))
    _close(g["mass"][bi], _fd(lambda x: O.rollout_loss(om, q0, v0, U, 5, w, mass=x, damping=damping, kp=kp), mass, bi))
    di = [0, 3, 6, 8, 14, 17]
    _close(g["damping"][di], _fd(lambda x: O.rollout_loss(om, q0, v0, U, 5, w, mass=mass, damping=x, kp=kp), damping, di))
    ki = list(range(12))
    _close(g["kp"][ki], _fd(lambda x: O.rollout_loss(om, q0, v0, U, 5, w, mass=mass, damping=damping, kp=x), kp, ki))


def test_gradient_at_rest_matches_central_differences():
    """A free body starting with zero angular velocity (a cylinder dropped upright onto a plane):
    the orientation update's derivative with respect to w at w = 0 (h / 2) must survive in reverse
    mode, else the tilt an angular-velocity perturbation causes is lost once contacts make the
    orientation matter."""
    b = W.ModelBuilder("upright")
    g0 = b.geom(0, W.PLANE, (0, 0, 0))
    body = b.body(0, (0, 0, 0.2))
    b.joint(body, W.FREE)
    g1 = b.geom(body, W.CYLINDER, (0.06, 0.1), mass=1.0)
    b.pair(g0, g1, friction=0.8, condim=3)
    m = b.build(timestep=0.002, iterations=100, n_substeps=4)
    om = O.OracleModel(m)
    w = O.tracking_loss_weights(om)
    q0 = np.array([-0.2, 0.0, 0.104, 1.0, 0.0, 0.0, 0.0])
    v0 = np.zeros(6)
    U = np.zeros((8, 0))
    g = O.rollout_grad(om, q0, v0, U, 4, w)
    fd = _fd(lambda x: O.rollout_loss(om, q0, x, U, 4, w), v0, range(6))
    _close(g["v0"], fd)
    assert abs(fd[4]) > 0.1


def test_step_vjp_chain_equals_rollout_gradient():
    """The per-control-step reverse sweep, chained along the trajectory with the loss cotangents,
    reproduces the rollout gradient (same tape, same order)."""
    m, om, q0, v0, U, w, mass = _setup(T=3, env=1)
    g = O.rollout_grad(om, q0, v0, U, m.n_substeps, w)
    wq, qs, wv, vs = w
    _, _, _, _, tq, tv = om.rollout(q0[None], v0[None], U[:, None], m.n_substeps, solver_cap=-1, trajectory=True)
    Q = np.concatenate([q0[None], tq[:, 0]]); V = np.concatenate([v0[None], tv[:, 0]])
    bq = np.zeros(m.nq); bv = np.zeros(m.nv); gm = np.zeros(m.nbody)
    for t in range(2, -1, -1):
        bq = bq + 2 * wq * (Q[t + 1] - qs); bv = bv + 2 * wv * (V[t + 1] - vs)
        o = O.step_vjp(om, Q[t], V[t], U[t], m.n_substeps, bq, bv)
        bq, bv = o["q"], o["v"]
        gm += o["mass"]
        assert np.allclose(o["u"], g["u"][t], rtol=1e-9, atol=1e-12)
    assert np.allclose(bq, g["q0"], rtol=1e-9, atol=1e-12)
    assert np.allclose(bv, g["v0"], rtol=1e-9, atol=1e-12)
    assert np.allclose(gm, g["mass"], rtol=1e-9, atol=1e-12)


def test_warm_started_resting_box_gradient_matches_central_differences():
    """A box dropped flat onto a plane comes to rest, and each substep's solve starts at the
    previous substep's minimiser (the warm start), so it converges on a step of rounding size.
    The taped gradient must still be the implicit derivative of the minimiser: against FP64
    central differences, with the lateral and spin components exactly zero by symmetry.  A tape
    that differentiates that last rounding-size step's line search instead was off by 1 % in
    v_x and gave the symmetric components 1e-3."""
    b = W.ModelBuilder("flat_box")
    g0 = b.geom(0, W.PLANE, (0, 0, 0))
    body = b.body(0, (0, 0, 0.2))
    b.joint(body, W.FREE)
    g1 = b.geom(body, W.BOX, (0.05, 0.05, 0.05), mass=1.0)
    b.pair(g0, g1, friction=0.8, condim=3)
    m = b.build(timestep=0.002, iterations=100, n_substeps=1)
    om = O.OracleModel(m)
    w = O.tracking_loss_weights(om)
    q0 = np.array([0.0, 0.0, 0.052, 1.0, 0.0, 0.0, 0.0])
    v0 = np.zeros(6)
    U = np.zeros((16, 0))
    g = O.rollout_grad(om, q0, v0, U, 1, w)
    fd = _fd(lambda x: O.rollout_loss(om, q0, x, U, 1, w), v0, range(6))
    _close(g["v0"], fd, rtol=1e-6)
    assert np.all(np.abs(g["v0"][[1, 3, 5]]) <= 1e-9)
    # the same horizon as 16 substeps inside one control step (warm starts taped)
    m16 = b.build(timestep=0.002, iterations=100, n_substeps=16)
    om16 = O.OracleModel(m16)
    g16 = O.rollout_grad(om16, q0, v0, np.zeros((1, 0)), 16, w)
    fd16 = _fd(lambda x: O.rollout_loss(om16, q0, x, np.zeros((1, 0)), 16, w), v0, range(6))
    _close(g16["v0"], fd16, rtol=1e-6)
