"""Pins of the oracle's joint friction loss (friction-loss rows: kind 3 of oracle/orc_step.hpp):
sliding deceleration and driven acceleration in closed form, the force bound, and the converged
Newton solve against a general minimiser on mixed rows."""
import numpy as np
import pytest
from scipy.optimize import minimize

from paper_2502_08844_b300 import workloads as W
from oracle import oracle as O


def _arm(F, kind=W.MOTOR):
    b = W.ModelBuilder("fric_arm")
    link = b.body(0, (0, 0, 0))
    b.joint(link, W.HINGE, axis=(0, 0, 1), frictionloss=F)
    b.geom(link, W.BOX, (0.2, 0.05, 0.05), pos=(0.2, 0, 0), mass=2.0)
    b.actuator(0, kind, gear=1.0)
    return b.build(timestep=0.002, gravity=(0, 0, 0), iterations=50)


def _inertia(om):
    return om.mass_matrix(np.zeros(1))[0, 0]


@pytest.mark.parametrize("v0", [2.0, -3.0])
def test_sliding_joint_decelerates_at_F_over_I(v0):
    """A spinning joint with friction loss F and no other force: while it slides, the row sits
    outside its band and the solve gives exactly a = -sign(v) F / I."""
    F = 0.3
    om = O.OracleModel(_arm(F))
    I = _inertia(om)
    f = om.forward(np.zeros(1), np.array([v0]), None, np.array([0.0]), solver_cap=-1)
    F32 = float(np.float32(F))                                           # the model's float32 value
    assert f["qacc"][0] == pytest.approx(-np.sign(v0) * F32 / I, rel=1e-12)
    assert abs(f["rows"][0, 1 + 6]) == pytest.approx(F32, rel=1e-12)    # the force sits at its bound


def test_driven_joint_accelerates_at_excess_torque():
    """A motor torque tau > F on a sliding joint: a = (tau - F) / I."""
    F, tau = 0.3, 1.1
    om = O.OracleModel(_arm(F))
    I = _inertia(om)
    f = om.forward(np.zeros(1), np.array([1.0]), None, np.array([tau]), solver_cap=-1)
    assert f["qacc"][0] == pytest.approx((tau - float(np.float32(F))) / I, rel=1e-12)


def test_friction_force_stays_within_its_bound_and_stops_the_joint():
    F = 0.4
    om = O.OracleModel(_arm(F))
    q, v = np.zeros((1, 1)), np.array([[1.5]])
    for _ in range(300):
        f = om.forward(q[0], v[0], None, np.array([0.0]), solver_cap=-1)
        assert abs(f["rows"][0, 1 + 6]) <= float(np.float32(F)) + 1e-12
        q, v, _, _ = om.rollout(q, v, np.zeros((1, 1, 1)), 1, solver_cap=-1)
    assert abs(v[0, 0]) < 1e-3          # stopped (the soft band leaves a vanishing creep)


def _cost(M, a0, J, aref, D, kind, mu, a):
    return O.cost(M, a0, J, aref, D, a, kind=kind, mu=mu)


def test_newton_matches_a_general_minimiser():
    rng = np.random.default_rng(3)
    for trial in range(20):
        nv, nr = 4, 6
        Q = rng.normal(size=(nv, nv))
        M = Q @ Q.T + nv * np.eye(nv)
        a0 = rng.normal(size=nv)
        J = rng.normal(size=(nr, nv))
        aref = rng.normal(size=nr)
        D = rng.uniform(0.5, 5.0, nr)
        kind = np.array([3, 3, 0, 3, 0, 3], np.int32)
        mu = np.where(kind == 3, rng.uniform(0.1, 2.0, nr), 0.0)
        a, force, it, conv = O.solve(M, a0, J, aref, D, cap=-1, kind=kind, mu=mu)
        assert conv
        res = minimize(lambda x: _cost(M, a0, J, aref, D, kind, mu, x), a0, method="BFGS",
                       options={"gtol": 1e-12, "maxiter": 2000})
        assert _cost(M, a0, J, aref, D, kind, mu, a) <= res.fun + 1e-10
        assert np.allclose(a, res.x, atol=1e-5)
        assert np.all(np.abs(force[kind == 3]) <= mu[kind == 3] + 1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_newton_with_elliptic_contacts_and_friction_loss_matches_a_general_minimiser(seed):
    """Friction-loss rows beside elliptic contacts (the elliptic hand with joint friction loss):
    the line search then walks the smooth convex phi(alpha), whose derivative takes each
    friction-loss row's D x inside its band and its bound +-F beyond.  The converged Newton solve
    equals BFGS on the same cost.  A line search that treats those rows as one-sided (a force only
    for x < 0) stops at the wrong alpha and fails here."""
    rng = np.random.default_rng(40 + seed)
    nv = 6
    Q = rng.normal(size=(nv, nv))
    M = Q @ Q.T + nv * np.eye(nv)
    a0 = rng.normal(size=nv) * 2
    kind = np.array([1, 2, 2, 3, 3, 1, 2, 2, 3], np.int32)
    nr = kind.size
    J = rng.normal(size=(nr, nv))
    aref = rng.normal(size=nr) * 3
    D = np.r_[[1.3] * 3, rng.uniform(0.5, 4.0, 2), [0.7] * 3, rng.uniform(0.5, 4.0, 1)]
    mu = np.r_[[0.9] * 3, rng.uniform(0.1, 1.5, 2), [0.4] * 3, rng.uniform(0.1, 1.5, 1)]
    a, force, it, conv = O.solve(M, a0, J, aref, D, cap=-1, kind=kind, mu=mu)
    assert conv
    f = lambda x: _cost(M, a0, J, aref, D, kind, mu, x)
    res = minimize(f, a0, method="BFGS", options={"gtol": 1e-12, "maxiter": 10000})
    assert f(a) <= res.fun + 1e-10 * (1 + abs(res.fun))
    np.testing.assert_allclose(a, res.x, rtol=1e-5, atol=1e-6)
    fr = kind == 3
    assert np.all(np.abs(force[fr]) <= mu[fr] + 1e-12)
