"""Pins of the oracle's elliptic friction cone.

The soft cost of an elliptic contact is half D times the squared distance from its residual
x = J a - aref to the dual cone K* = {x_n >= mu |x_t|}.  The pins check five things:

* the cost against a projection computed by a general constrained solver (SLSQP);
* gradient and Hessian against finite differences;
* the Newton solve against a general minimiser of the same cost;
* the isotropy of sliding friction (the pyramid is not isotropic), with |f_t| = mu f_n;
* the 5/7 rolling law.

CPU only."""
import dataclasses

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import oracle as O
from paper_2502_08844_b300 import workloads as W
from tests import models_for_tests as TM


def _project_dual_cone(x, mu):
    """Euclidean projection onto {y_n >= mu |y_t|} by SLSQP (independent of the closed form)."""
    cons = {"type": "ineq", "fun": lambda y: y[0] - mu * np.sqrt(y[1] ** 2 + y[2] ** 2 + 1e-300)}
    best = None
    for y0 in (np.array([abs(x[0]) + mu * np.linalg.norm(x[1:]) + 1.0, x[1], x[2]]), np.zeros(3) + [1e-3, 0, 0]):
        r = minimize(lambda y: np.sum((y - x) ** 2), y0, constraints=[cons], method="SLSQP",
                     options={"ftol": 1e-15, "maxiter": 500})
        if best is None or r.fun < best.fun:
            best = r
    return best.x


@pytest.mark.parametrize("seed", range(6))
def test_cone_cost_is_half_D_squared_distance_to_dual_cone(seed):
    rng = np.random.default_rng(seed)
    mu, D = rng.uniform(0.3, 1.5), rng.uniform(0.5, 3.0)
    for _ in range(20):
        x = rng.normal(size=3) * rng.uniform(0.1, 3.0)
        f, g, H, zone = O.cone_cost(x, D, mu)
        y = _project_dual_cone(x, mu)
        ref = 0.5 * D * np.sum((x - y) ** 2)
        assert f == pytest.approx(ref, rel=1e-6, abs=1e-9), (x, zone)
        # the force -grad s = -D (x - P(x)) lies in the friction cone K = {|f_t| <= mu f_n}
        fn, ft = -g[0], np.linalg.norm(g[1:])
        assert fn >= -1e-12 and ft <= mu * fn + 1e-9


def test_cone_gradient_and_hessian_match_finite_differences():
    rng = np.random.default_rng(5)
    mu, D, h = 0.8, 1.7, 1e-6
    zones = set()
    for _ in range(60):
        x = rng.normal(size=3)
        f, g, H, z = O.cone_cost(x, D, mu)
        zones.add(z)
        for i in range(3):
            e = np.zeros(3); e[i] = h
            fp, gp, _, zp = O.cone_cost(x + e, D, mu)
            fm, gm, _, zm = O.cone_cost(x - e, D, mu)
            if zp != z or zm != z:
                continue   # a zone boundary inside the stencil
            assert (fp - fm) / (2 * h) == pytest.approx(g[i], rel=1e-6, abs=1e-8)
            np.testing.assert_allclose((gp - gm) / (2 * h), H[:, i], rtol=1e-5, atol=1e-6)
    assert zones == {0, 1, 2}


@pytest.mark.parametrize("seed", range(5))
def test_elliptic_newton_reaches_the_minimiser(seed):
    """Two elliptic contacts and a scalar row on a random convex problem: the converged Newton
    solve equals a general minimiser (BFGS) of the same cost."""
    rng = np.random.default_rng(100 + seed)
    nv = 6
    A = rng.normal(size=(nv, nv))
    M = A @ A.T + nv * np.eye(nv)
    a0 = rng.normal(size=nv)
    J = rng.normal(size=(7, nv))
    aref = rng.normal(size=7) * 3
    D = np.r_[[1.3] * 3, [0.7] * 3, 2.0]
    kind = [1, 2, 2, 1, 2, 2, 0]
    mu = [0.9] * 3 + [0.4] * 3 + [0.0]
    q, force, it, conv = O.solve(M, a0, J, aref, D, cap=-1, kind=kind, mu=mu)
    assert conv
    f = lambda a: O.cost(M, a0, J, aref, D, a, kind=kind, mu=mu)
    r = minimize(f, a0, method="BFGS", options={"gtol": 1e-11, "maxiter": 10000})
    assert f(q) <= r.fun + 1e-10 * (1 + abs(r.fun))
    np.testing.assert_allclose(q, r.x, rtol=1e-5, atol=1e-6)


def _sliding_sphere_forces(cone, theta, mu=0.5, speed=0.4):
    m = dataclasses.replace(TM.sphere_on_plane(mass=1.0, radius=0.1, friction=mu, condim=3), cone=cone)
    om = O.OracleModel(m)
    r = float(np.float32(0.1))
    q = np.array([0, 0, r - 1e-4, 1, 0, 0, 0.0])
    v = np.array([speed * np.cos(theta), speed * np.sin(theta), 0, 0, 0, 0.0])
    rec = om.forward(q, v, solver_cap=-1)
    rows = rec["rows"][: rec["nrow"]]
    return rows[:, m.nv:], rec


def test_elliptic_sliding_friction_is_isotropic_and_on_the_cone():
    mu = 0.5
    out = []
    for theta in (0.0, np.pi / 6, np.pi / 4, 1.0):
        rows, rec = _sliding_sphere_forces(W.ELLIPTIC, theta, mu)
        assert rows.shape[0] == 3
        f = rows[:, 6]   # (n, t1, t2) force
        assert f[0] > 0
        assert np.hypot(f[1], f[2]) == pytest.approx(mu * f[0], rel=1e-9)   # sliding: on the cone
        # in world axes (the contact's t1, t2) friction opposes the sliding direction
        con = rec["contacts"][0]
        fw = f[1] * con[8:11] + f[2] * con[11:14]
        np.testing.assert_allclose(fw[:2] / np.linalg.norm(fw), [-np.cos(theta), -np.sin(theta)], atol=1e-9)
        out.append(f[0])
    np.testing.assert_allclose(out, out[0], rtol=1e-9)
    # the pyramid is not isotropic: diagonal sliding gets a different friction magnitude
    rows0, _ = _sliding_sphere_forces(W.PYRAMIDAL, 0.0, mu)
    rows45, _ = _sliding_sphere_forces(W.PYRAMIDAL, np.pi / 4, mu)
    assert abs(np.abs(rows0[:, 6]).sum() - np.abs(rows45[:, 6]).sum()) > 1e-3 * np.abs(rows0[:, 6]).sum()


def test_elliptic_sliding_sphere_ends_rolling_at_five_sevenths():
    m = dataclasses.replace(TM.sphere_on_plane(mass=1.0, radius=0.1, friction=1.0, condim=3, timestep=0.002),
                            cone=W.ELLIPTIC)
    om = O.OracleModel(m)
    v0 = 0.05
    q = np.array([[0, 0, 0.1, 1, 0, 0, 0]]); v = np.array([[0.6 * v0, 0.8 * v0, 0, 0, 0, 0]])
    q2, v2, _, _ = om.rollout(q, v, np.zeros((1000, 1, 0)), 1)
    vt = np.hypot(v2[0, 0], v2[0, 1])
    assert vt == pytest.approx(5.0 / 7.0 * v0, rel=3e-3)
    assert np.arctan2(v2[0, 1], v2[0, 0]) == pytest.approx(np.arctan2(0.8, 0.6), abs=1e-6)
