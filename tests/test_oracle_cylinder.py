"""Pins of the oracle's cylinder: its inertia against grid integration, its contact points against
brute force over the rims, and statics and rolling against closed forms."""
import math

import numpy as np
import pytest

from paper_2502_08844_b300 import workloads as W
from oracle import oracle as O


def _rot(q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_cylinder_inertia_matches_grid_integration():
    r, hl, m = 0.07, 0.12, 1.3
    n = 240
    lo, hi = [-r, -r, -hl], [r, r, hl]
    axes = [np.linspace(lo[k], hi[k], n, endpoint=False) + (hi[k] - lo[k]) / (2 * n) for k in range(3)]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    mask = X ** 2 + Y ** 2 <= r * r
    cnt = mask.sum()
    I = m * np.array([((Y ** 2 + Z ** 2) * mask).sum(), ((X ** 2 + Z ** 2) * mask).sum(),
                      ((X ** 2 + Y ** 2) * mask).sum()]) / cnt
    assert np.allclose(O.solid_inertia(W.CYLINDER, (r, hl), m), I, rtol=1e-2)


def _plane_cyl(R2, p2, r=0.1, hl=0.25, nrm=(0.0, 0.0, 1.0)):
    n = np.asarray(nrm, np.float64)
    n = n / np.linalg.norm(n)
    # plane frame with z along n
    t = np.cross(n, [1.0, 0, 0]) if abs(n[0]) < 0.9 else np.cross(n, [0, 1.0, 0])
    t /= np.linalg.norm(t)
    R1 = np.stack([t, np.cross(n, t), n], 1)
    p1 = np.array([0.1, -0.2, 0.05])
    return O.collide(W.PLANE, R1, p1, (0, 0, 0), W.CYLINDER, R2, p2, (r, hl)), n, p1


def _rim(R2, p2, r, hl, side, k=20000):
    th = np.linspace(0, 2 * np.pi, k, endpoint=False)
    loc = np.stack([r * np.cos(th), r * np.sin(th), np.full(k, side * hl)], 1)
    return p2 + loc @ R2.T


@pytest.mark.parametrize("seed", range(6))
def test_deepest_points_match_brute_force_over_the_rims(seed):
    """Slot 0 is the deepest point of the whole solid (a point of a rim circle), slot 1 the deepest
    point of the other rim; slots 2 and 3 lie on the first rim 120 degrees either side of slot 0."""
    rng = np.random.default_rng(seed)
    R2 = _rot(rng.normal(size=4))
    p2 = rng.normal(0, 0.1, 3) + [0, 0, 0.2]
    r, hl = 0.1, 0.25
    c, n, p1 = _plane_cyl(R2, p2, r, hl, nrm=rng.normal(size=3) * [0.2, 0.2, 1] + [0, 0, 2])
    assert c.shape == (4, 13)
    depth = lambda P: (P - p1) @ n
    rims = [depth(_rim(R2, p2, r, hl, s)) for s in (-1, 1)]
    lo = int(np.argmin([x.min() for x in rims]))
    # the solid's deepest point over a plane is a rim point (a linear function on a convex set
    # takes its minimum at an extreme point; the extreme points of a cylinder are its rims)
    assert c[0, 0] == pytest.approx(rims[lo].min(), abs=1e-8)
    assert c[1, 0] == pytest.approx(rims[1 - lo].min(), abs=1e-8)
    a = R2[:, 2]
    cap = p2 + (2 * lo - 1) * hl * a
    pts = [c[k, 1:4] + c[k, 0] / 2 * n for k in range(4)]          # the rim points themselves
    for k in range(4):
        assert np.allclose(c[k, 4:7], n, atol=1e-14)
    u = [(pts[k] - cap) for k in (0, 2, 3)]
    for v in u:
        assert np.linalg.norm(v) == pytest.approx(r, rel=1e-12) and abs(v @ a) < 1e-12
    for v in u[1:]:
        assert math.degrees(math.acos(np.clip(v @ u[0] / r ** 2, -1, 1))) == pytest.approx(120.0, abs=1e-9)
    assert c[2, 0] == pytest.approx(c[3, 0], abs=1e-12) and c[2, 0] >= c[0, 0]


def test_standing_cylinder_points_form_a_tripod():
    r, hl = 0.1, 0.25
    c, n, p1 = _plane_cyl(np.eye(3), np.array([0.3, 0.0, 0.05 + hl - 0.001]), r, hl)
    for k in (0, 2, 3):
        assert c[k, 0] == pytest.approx(-0.001, abs=1e-14)
    assert c[1, 0] == pytest.approx(2 * hl - 0.001, abs=1e-14)
    # the three lower points sit on the rim 120 degrees apart, the first along the cylinder's x axis
    pts = np.array([c[k, 1:3] for k in (0, 2, 3)]) - [0.3, 0.0]
    assert np.allclose(pts[0], [r, 0], atol=1e-14)
    assert np.allclose(np.linalg.norm(pts, axis=1), r, atol=1e-14)


def _cylinder_model(quat, z, friction=1.0, gravity=(0, 0, -9.81), condim=3):
    b = W.ModelBuilder("cyl")
    g0 = b.geom(0, W.PLANE, (0, 0, 0))
    body = b.body(0, (0, 0, z))
    b.joint(body, W.FREE)
    g1 = b.geom(body, W.CYLINDER, (0.1, 0.25), quat=quat, mass=2.0)
    b.pair(g0, g1, friction=friction, condim=condim)
    return b.build(timestep=0.002, iterations=50, gravity=gravity)


def _settle(m, q0, steps=1500):
    om = O.OracleModel(m)
    q = np.asarray(q0, np.float64)[None]
    v = np.zeros((1, 6))
    q, v, _, _ = om.rollout(q, v, np.zeros((steps, 1, 0)), 1, solver_cap=-1)
    return om, q[0], v[0]


def _edge_normal_forces(om, q, v, per_contact=4):
    f = om.forward(q, v, np.zeros(6), None, solver_cap=-1)
    rows = f["rows"]
    nv = om.nv
    # each active contact contributes 4 pyramid edge rows (1 row when frictionless); their
    # normal components add up
    return rows[:, nv + 6].reshape(-1, per_contact).sum(1), f


def test_standing_cylinder_rests_on_three_equal_contacts():
    """Standing on a cap, the cylinder comes to rest on its tripod; the three normal forces must
    add up to m g with their centroid under the centre of mass, so each carries m g / 3.  The
    contact is frictionless here: with pyramid friction each edge row's D follows its own A-hat,
    and on a three-fold contact set that leaves a small steady creep (about 4e-4 m/s), a property
    of the soft pyramidal model rather than of the contact points."""
    m = _cylinder_model((1, 0, 0, 0), 0.25, condim=1)
    om, q, v = _settle(m, [0, 0, 0.25, 1, 0, 0, 0])
    assert np.abs(v).max() < 1e-6
    fn, _ = _edge_normal_forces(om, q, v, per_contact=1)
    assert len(fn) == 3
    assert np.allclose(fn, 2.0 * 9.81 / 3, rtol=1e-6)


def test_lying_cylinder_rests_on_its_two_rims():
    s = math.sqrt(0.5)
    m = _cylinder_model((s, s, 0, 0), 0.1)           # axis along y
    om, q, v = _settle(m, [0, 0, 0.1, 1, 0, 0, 0])
    assert np.abs(v).max() < 1e-6
    fn, _ = _edge_normal_forces(om, q, v)
    assert len(fn) == 2 and np.allclose(fn, 2.0 * 9.81 / 2, rtol=1e-6)


def test_cylinder_rolls_down_an_incline_at_two_thirds_g_sin():
    """A solid cylinder rolling without slipping down a slope of angle th accelerates at
    g sin(th) / (1 + I / (m r^2)) = (2/3) g sin(th)."""
    th = 0.2
    g = 9.81
    s = math.sqrt(0.5)
    m = _cylinder_model((s, s, 0, 0), 0.1, friction=1.0, gravity=(g * math.sin(th), 0, -g * math.cos(th)))
    om = O.OracleModel(m)
    q = np.array([[0, 0, 0.0995, 1, 0, 0, 0]])
    v = np.zeros((1, 6))
    q1, v1, _, _ = om.rollout(q, v, np.zeros((250, 1, 0)), 1, solver_cap=-1)
    q2, v2, _, _ = om.rollout(q1, v1, np.zeros((250, 1, 0)), 1, solver_cap=-1)
    acc = (v2[0, 0] - v1[0, 0]) / (250 * 0.002)
    assert acc == pytest.approx(2.0 / 3.0 * g * math.sin(th), rel=3e-3)
    assert abs(v2[0, 0] - 0.1 * v2[0, 4]) < 3e-3 * abs(v2[0, 0])       # rolling: v = r w


def test_plane_cylinder_is_the_only_cylinder_pair():
    with pytest.raises(ValueError):
        O.collide(W.SPHERE, np.eye(3), np.zeros(3), (0.1,), W.CYLINDER, np.eye(3), np.ones(3), (0.1, 0.2))
