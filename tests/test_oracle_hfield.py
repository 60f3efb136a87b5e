"""Pins of the oracle's heightfield collision (oracle/orc_step.hpp hfield_sphere) against planes
it must reduce to, a brute-force minimum over every triangle by a general QP solver, and frame
changes; and of its use inside the model (a ball dropped on a flat heightfield moves as on the
equivalent plane)."""
import math

import numpy as np
import pytest
from scipy.optimize import minimize

from paper_2502_08844_b300 import workloads as W
from oracle import oracle as O

I3 = np.eye(3)
SIZE = np.array([1.0, 0.8, 0.1])    # hx, hy, hz


def _rz(psi):
    c, s = math.cos(psi), math.sin(psi)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])


def _hf(elev, c, r, R1=I3, p1=(0, 0, 0)):
    return O.collide_hfield(R1, p1, SIZE, elev, W.SPHERE, I3, c, [r])[0]


def _grid(fn, nrow=9, ncol=11):
    y = np.linspace(-SIZE[1], SIZE[1], nrow)
    x = np.linspace(-SIZE[0], SIZE[0], ncol)
    Y, X = np.meshgrid(y, x, indexing="ij")
    return fn(X, Y)


def test_flat_grid_is_a_plane():
    elev = _grid(lambda X, Y: np.full_like(X, 0.4))
    rng = np.random.default_rng(0)
    for _ in range(50):
        c = np.array([rng.uniform(-0.95, 0.95), rng.uniform(-0.75, 0.75), 0.04 + rng.uniform(-0.03, 0.03)])
        r = 0.02
        h = _hf(elev, c, r)
        p = O.collide(W.PLANE, I3, [0, 0, 0.04], [0, 0, 0], W.SPHERE, I3, c, [r])[0]
        assert np.allclose(h[:7], p[:7], atol=1e-12)


def test_tilted_planar_grid_is_an_inclined_plane():
    """Elevations linear in x make every triangle lie in one plane z = a + b x."""
    a, b = 0.05, 0.03                     # surface height 0.1 * e = a + b x
    elev = _grid(lambda X, Y: (a + b * X) / SIZE[2])
    n = np.array([-b, 0.0, 1.0]) / math.hypot(b, 1.0)
    rng = np.random.default_rng(1)
    for _ in range(50):
        x, y = rng.uniform(-0.8, 0.8), rng.uniform(-0.6, 0.6)
        c = np.array([x, y, a + b * x + rng.uniform(0.0, 0.03)])
        r = 0.025
        h = _hf(elev, c, r)
        s = n @ (c - np.array([0.0, 0.0, a]))
        assert h[0] == pytest.approx(s - r, abs=1e-12)
        assert np.allclose(h[4:7], n, atol=1e-9)
        assert np.allclose(h[1:4], c - n * (r + (s - r) / 2), atol=1e-12)


def _triangles(elev):
    nrow, ncol = elev.shape
    xs = np.linspace(-SIZE[0], SIZE[0], ncol)
    ys = np.linspace(-SIZE[1], SIZE[1], nrow)
    V = lambda i, j: np.array([xs[j], ys[i], SIZE[2] * elev[i, j]])
    for i in range(nrow - 1):
        for j in range(ncol - 1):
            yield V(i, j), V(i, j + 1), V(i + 1, j + 1)
            yield V(i, j), V(i + 1, j + 1), V(i + 1, j)


def _qp_distance(p, tri):
    """Distance from p to a triangle by SLSQP over barycentric weights (a general solver)."""
    a, b, c = tri
    f = lambda w: np.sum((a + w[0] * (b - a) + w[1] * (c - a) - p) ** 2)
    cons = [{"type": "ineq", "fun": lambda w: 1.0 - w[0] - w[1]}]
    best = min((minimize(f, w0, method="SLSQP", bounds=[(0, 1), (0, 1)], constraints=cons,
                         options={"ftol": 1e-16, "maxiter": 200}) for w0 in ([1 / 3, 1 / 3], [0.05, 0.05])),
               key=lambda res: res.fun)
    return math.sqrt(max(best.fun, 0.0))


def test_rough_grid_matches_the_minimum_over_every_triangle():
    rng = np.random.default_rng(2)
    elev = rng.uniform(0, 1, (7, 8))
    tris = list(_triangles(elev))
    hits = 0
    for _ in range(25):
        x, y = rng.uniform(-0.9, 0.9), rng.uniform(-0.7, 0.7)
        r = 0.06
        c = np.array([x, y, 0.0])
        c[2] = SIZE[2] * np.max(elev) + 0.02 if rng.uniform() < 0.3 else SIZE[2] * np.interp(x, np.linspace(-1, 1, 8), elev[3]) + 0.05
        h = _hf(elev, c, r)
        near = [t for t in tris if min(np.min(np.abs(np.array(t)[:, :2] - c[:2]).max(axis=1)), 1.0) < 0.5]
        dmin = min(_qp_distance(c, t) for t in near)
        if dmin < r:                       # a contact: the local search found the global minimum
            hits += 1
            assert h[0] == pytest.approx(dmin - r, abs=1e-7)
        else:
            assert h[0] >= -1e-9           # no contact either way
    assert hits >= 5


def test_rotated_and_shifted_grid():
    """A yawed, shifted heightfield gives the contacts of the unrotated grid in its own frame."""
    rng = np.random.default_rng(3)
    elev = rng.uniform(0, 1, (6, 6))
    R1, p1 = _rz(0.7), np.array([0.3, -0.2, 0.05])
    for _ in range(20):
        cl = np.array([rng.uniform(-0.9, 0.9), rng.uniform(-0.7, 0.7), rng.uniform(0.05, 0.12)])
        h0 = _hf(elev, cl, 0.05)
        h1 = _hf(elev, R1 @ cl + p1, 0.05, R1, p1)
        assert h1[0] == pytest.approx(h0[0], abs=1e-12)
        assert np.allclose(h1[4:7], R1 @ h0[4:7], atol=1e-12)
        assert np.allclose(h1[1:4], R1 @ h0[1:4] + p1, atol=1e-12)


def test_outside_and_deep_cases():
    elev = _grid(lambda X, Y: 0.5 + 0.3 * X)
    assert _hf(elev, np.array([1.2, 0.0, 0.05]), 0.02)[0] >= 1e29           # off the footprint
    c = np.array([0.2, 0.1, 0.0])                                           # below the surface z = 0.05 + 0.03 x
    h = _hf(elev, c, 0.02)
    n = np.array([-0.03, 0.0, 1.0]) / math.hypot(0.03, 1.0)
    s = n @ (c - np.array([0.0, 0.0, 0.05]))
    assert s < 0 and h[0] == pytest.approx(s - 0.02, abs=1e-12) and np.allclose(h[4:7], n)


def test_capsule_meets_the_terrain_at_its_end_spheres():
    rng = np.random.default_rng(4)
    elev = rng.uniform(0, 1, (6, 7))
    R2 = np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0.0]])    # capsule axis along world y
    p2 = np.array([0.1, 0.05, 0.09])
    out = O.collide_hfield(I3, [0, 0, 0], SIZE, elev, W.CAPSULE, R2, p2, [0.03, 0.2])
    assert out.shape[0] == 2
    for e, sg in enumerate((-1, 1)):
        assert np.allclose(out[e], _hf(elev, p2 + sg * 0.2 * R2[:, 2], 0.03), atol=1e-14)


def _ball(floor_type, size, hfield=None, z0=0.3):
    b = W.ModelBuilder("ball")
    g0 = b.geom(0, floor_type, size)
    ball = b.body(0, (0, 0, z0))
    b.joint(ball, W.FREE)
    g1 = b.geom(ball, W.SPHERE, (0.05,), mass=1.0)
    b.pair(g0, g1, friction=1.0, condim=3)
    return b.build(timestep=0.002, iterations=50, hfield=hfield)


def test_ball_on_a_flat_heightfield_moves_as_on_the_plane():
    """The same ball thrown onto a flat heightfield at height 0.04 and onto the plane z = 0.04
    (the plane's geom raised by 0.04): identical trajectories, sliding and coming to rest."""
    flat = np.full((5, 5), 0.4, np.float32)
    mh = _ball(W.HFIELD, (2.0, 2.0, 0.1), hfield=flat)
    mp = _ball(W.PLANE, (0, 0, 0))
    mp.geom_pos = mp.geom_pos.copy(); mp.geom_pos[0, 2] = np.float32(0.04)
    oh, op = O.OracleModel(mh), O.OracleModel(mp)
    q = np.array([[0.1, -0.2, 0.2, 1, 0, 0, 0]]); v = np.array([[1.0, 0.5, 0.0, 0.0, 3.0, 0.0]])
    u = np.zeros((400, 1, 0))
    qh, vh, _, _ = oh.rollout(q, v, u, 1, solver_cap=-1)
    qp, vp, _, _ = op.rollout(q, v, u, 1, solver_cap=-1)
    assert np.allclose(qh, qp, atol=1e-10) and np.allclose(vh, vp, atol=1e-10)
    assert qh[0, 2] == pytest.approx(0.04 + 0.05, abs=2e-3)      # resting on the surface
