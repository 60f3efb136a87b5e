"""Pins of the oracle's convex meshes and solid contacts (plane against a mesh, heightfield against
a box or a mesh): mass properties against closed forms and grid integration, contacts against the
box-plane routine, planar heightfields against planes, a terrain spike inside a box in closed
form, a vertex's depth against the terrain height interpolated in its triangle, and a resting hull
against statics."""
import dataclasses

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2502_08844_b300 import workloads as W

PLANE, BOX, HFIELD, MESH = W.PLANE, W.BOX, W.HFIELD, W.MESH


def _box_mesh(h, offset=(0.0, 0.0, 0.0)):
    """a box of half sizes h as a mesh: corners (bit k of i chooses + on axis k), 12 outward triangles"""
    v = np.array([[(h[0] if i & 1 else -h[0]), (h[1] if i & 2 else -h[1]), (h[2] if i & 4 else -h[2])] for i in range(8)])
    quads = [(0, 4, 6, 2), (1, 3, 7, 5), (0, 1, 5, 4), (2, 6, 7, 3), (0, 2, 3, 1), (4, 5, 7, 6)]
    f = []
    for a, b, c, d in quads:
        f += [(a, b, c), (a, c, d)]
    f = np.array(f)
    for t in f:   # outward
        n = np.cross(v[t[1]] - v[t[0]], v[t[2]] - v[t[0]])
        assert np.dot(n, v[t[0]]) > 0
    return v + np.asarray(offset), f


def _octahedron(a):
    v = np.array([[a, 0, 0], [-a, 0, 0], [0, a, 0], [0, -a, 0], [0, 0, a], [0, 0, -a]], float)
    f = []
    for sx in (0, 1):
        for sy in (2, 3):
            for sz in (4, 5):
                t = [sx, sy, sz]
                if np.dot(np.cross(v[t[1]] - v[t[0]], v[t[2]] - v[t[0]]), v[t[0]] + v[t[1]] + v[t[2]]) < 0:
                    t = [sx, sz, sy]
                f.append(t)
    return v, np.array(f)


def _one_body(vert, face, mass, pos=(0, 0, 0), quat=(1, 0, 0, 0)):
    b = W.ModelBuilder("one_mesh")
    body = b.body(0, (0, 0, 1))
    b.joint(body, W.FREE)
    mk = b.mesh(vert, face)
    b.geom(body, MESH, (0, 0, 0), pos=pos, quat=quat, mass=mass, mesh=mk)
    return b.build(timestep=0.002)


def _massprops(m):
    mass, ipos, inertia, _ = O.OracleModel(m).massprops()
    I = inertia[1]
    return mass[1], ipos[1], np.array([[I[0], I[3], I[4]], [I[3], I[1], I[5]], [I[4], I[5], I[2]]])


def test_box_mesh_has_the_box_mass_properties():
    """a box as a mesh, offset from its geom frame and the geom rotated: the centre of mass moves
    with the offset and the inertia is the box's (m/12 (b^2 + c^2) ...) rotated.  A dropped
    parallel-axis shift or a transposed rotation fails it."""
    h = (0.2, 0.1, 0.05)
    off = np.array([0.03, -0.02, 0.01])
    q = Rotation.from_euler("xyz", [0.3, -0.2, 0.5]).as_quat()[[3, 0, 1, 2]]
    v, f = _box_mesh(h, off)
    m = _one_body(v, f, 2.0, pos=(0.1, 0.0, -0.05), quat=q)
    M, c, I = _massprops(m)
    R = Rotation.from_quat(q[[1, 2, 3, 0]]).as_matrix()
    a, b, cc = 2 * np.array(h)
    Ib = np.diag([2.0 / 12 * (b * b + cc * cc), 2.0 / 12 * (a * a + cc * cc), 2.0 / 12 * (a * a + b * b)])
    assert M == pytest.approx(2.0, rel=1e-12)
    np.testing.assert_allclose(c, np.array([0.1, 0.0, -0.05]) + R @ off, atol=1e-7)   # float32 inputs
    np.testing.assert_allclose(I, R @ Ib @ R.T, rtol=1e-5, atol=1e-9)


def test_octahedron_inertia_in_closed_form():
    """|x| + |y| + |z| <= a: each axis m a^2 / 5 (the second moment per unit mass is a^2 / 10)."""
    v, f = _octahedron(0.1)
    M, c, I = _massprops(_one_body(v, f, 3.0))
    np.testing.assert_allclose(c, 0, atol=1e-12)
    np.testing.assert_allclose(I, np.eye(3) * 3.0 * 0.01 / 5, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("seed", [101, 102, 103])
def test_hull_mass_properties_against_grid_integration(seed):
    """a seeded hull: volume-weighted centre and inertia against a midpoint-rule integration over a
    120^3 grid of its inside (points inside every face plane, the planes from the test's own
    cross products)."""
    v, f = W.convex_hull(seed, 16, (0.08, 0.05, 0.06))
    M, c, I = _massprops(_one_body(v, f, 1.0))
    lo, hi = v.min(0), v.max(0)
    n = 120
    axes = [lo[k] + (np.arange(n) + 0.5) * (hi[k] - lo[k]) / n for k in range(3)]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    inside = np.ones(len(P), bool)
    for t in f:
        nrm = np.cross(v[t[1]] - v[t[0]], v[t[2]] - v[t[0]])
        inside &= (P - v[t[0]]) @ nrm <= 0
    Q = P[inside]
    com = Q.mean(0)
    d = Q - com
    Ig = (np.eye(3) * (d * d).sum(1).mean() - d.T @ d / len(d)) * 1.0
    np.testing.assert_allclose(c, com, atol=2e-4)
    np.testing.assert_allclose(I, Ig, rtol=0.02, atol=2e-2 * np.abs(Ig).max())


def _rand_pose(rng, z):
    R = Rotation.from_euler("xyz", rng.uniform(-0.6, 0.6, 3)).as_matrix()
    return R, np.array([rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), z])


@pytest.mark.parametrize("seed", range(6))
def test_plane_mesh_equals_plane_box_for_a_box_mesh(seed):
    """the box-plane routine (its own corner loop) and the mesh routine on the box as a mesh give
    the same 4 contacts in the same order"""
    rng = np.random.default_rng(seed)
    h = (0.15, 0.1, 0.05)
    v, f = _box_mesh(h)
    R1 = Rotation.from_euler("xyz", rng.uniform(-0.2, 0.2, 3)).as_matrix()
    p1 = rng.uniform(-0.1, 0.1, 3)
    R2, p2 = _rand_pose(rng, p1[2] + 0.06)
    ref = O.collide(PLANE, R1.ravel(), p1, (0, 0, 0), BOX, R2.ravel(), p2, h)
    got = O.collide_mesh(R1.ravel(), p1, R2.ravel(), p2, v, f)
    np.testing.assert_allclose(got, ref, atol=1e-12)


def _grid(nrow, ncol, fn):
    i, j = np.meshgrid(np.arange(nrow), np.arange(ncol), indexing="ij")
    return fn(i / (nrow - 1), j / (ncol - 1))


@pytest.mark.parametrize("seed", range(4))
def test_box_on_flat_grid_equals_box_on_plane(seed):
    """a flat grid (every elevation 0.5, hz 0.2: a plane at z = 0.1) with vertices 2 m apart, none
    under the box: the box's contacts are the box-plane ones"""
    rng = np.random.default_rng(10 + seed)
    h = (0.15, 0.1, 0.05)
    elev = _grid(3, 3, lambda a, b: 0.5 + 0 * a)
    size = (2.0, 2.0, 0.2)
    R2, p2 = _rand_pose(rng, 0.1 + 0.06)
    p2[:2] += (0.7, 0.5)
    I3 = np.eye(3).ravel()
    got = O.collide_mesh(I3, np.zeros(3), R2.ravel(), p2, *_box_mesh(h), size=size, elev=elev)
    ref = O.collide(PLANE, I3, np.array([0, 0, 0.1]), (0, 0, 0), BOX, R2.ravel(), p2, h)
    np.testing.assert_allclose(got, ref, atol=1e-12)
    box = O.collide_hfield(I3, np.zeros(3), size, elev, BOX, R2.ravel(), p2, h)   # the box's own solid
    np.testing.assert_allclose(box, ref, atol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_box_on_planar_slope_equals_box_on_inclined_plane(seed):
    """elevations linear in x (0 at x = -hx, 1 at x = +hx, hz 0.4 over 4 m: slope 0.1): every
    triangle is the inclined plane, so a box's contacts are the box-plane ones on that plane"""
    rng = np.random.default_rng(20 + seed)
    h = (0.15, 0.1, 0.05)
    size = (2.0, 2.0, 0.4)
    elev = _grid(3, 3, lambda a, b: b + 0 * a)
    nrm = np.array([-0.4 / 4.0, 0.0, 1.0])
    nrm /= np.linalg.norm(nrm)
    x0, y0 = 0.7, 0.5
    z0 = 0.4 * (x0 + 2.0) / 4.0
    R2, p2 = _rand_pose(rng, 0.0)
    p2 += np.array([x0, y0, z0]) + 0.06 * nrm
    # the inclined plane's frame: its z axis along nrm
    Rp = Rotation.align_vectors([nrm], [[0, 0, 1]])[0].as_matrix()
    I3 = np.eye(3).ravel()
    got = O.collide_mesh(I3, np.zeros(3), R2.ravel(), p2, *_box_mesh(h), size=size, elev=elev)
    ref = O.collide(PLANE, Rp.ravel(), np.array([x0, y0, z0]), (0, 0, 0), BOX, R2.ravel(), p2, h)
    np.testing.assert_allclose(got[:, :7], ref[:, :7], atol=1e-12)   # dist, pos, normal
    box = O.collide_hfield(I3, np.zeros(3), size, elev, BOX, R2.ravel(), p2, h)
    np.testing.assert_allclose(box[:, :7], ref[:, :7], atol=1e-12)


def test_terrain_spike_inside_a_box():
    """a 3 x 3 grid, flat at 0 but for its centre vertex at 0.1, under an axis-aligned box whose
    bottom face lies at 0.08: the spike is the one penetrating candidate, 2 cm deep, normal +z
    (minus the bottom face's outward normal), midway between the tip and the face"""
    size = (1.0, 1.0, 0.1)
    elev = np.zeros((3, 3)); elev[1, 1] = 1.0
    h = (0.3, 0.3, 0.05)
    p2 = np.array([0.0, 0.0, 0.13])
    I3 = np.eye(3).ravel()
    got = O.collide_mesh(I3, np.zeros(3), I3, p2, *_box_mesh(h), size=size, elev=elev)
    np.testing.assert_allclose(O.collide_hfield(I3, np.zeros(3), size, elev, BOX, I3, p2, h), got, atol=1e-12)
    act = got[got[:, 0] < 0]
    assert len(act) == 1
    assert act[0, 0] == pytest.approx(-0.02, abs=1e-12)
    np.testing.assert_allclose(act[0, 4:7], [0, 0, 1], atol=1e-12)
    np.testing.assert_allclose(act[0, 1:4], [0, 0, 0.09], atol=1e-12)
    assert got[3, 0] == act[0, 0]   # after the 3 shallowest corners (candidate order)


@pytest.mark.parametrize("seed", range(5))
def test_vertex_depth_is_its_height_over_the_terrain_along_the_triangle_normal(seed):
    """a tetrahedron with one vertex pointing down into a bumpy grid: its deepest contact is that
    vertex, at nt_z (v_z - h(x, y)) with h the terrain height interpolated in the triangle under it
    (barycentric weights in the grid's xy) and nt its unit normal"""
    rng = np.random.default_rng(30 + seed)
    nr, nc = 6, 7
    elev = rng.uniform(0, 1, (nr, nc))
    size = (1.0, 1.2, 0.1)
    dx, dy = 2 * size[0] / (nc - 1), 2 * size[1] / (nr - 1)
    x, y = rng.uniform(-0.8, 0.8), rng.uniform(-1.0, 1.0)
    # the grid's own triangles: cell by floor, diagonal (i, j)-(i+1, j+1)
    j, i = int((x + size[0]) // dx), int((y + size[1]) // dy)
    fu, fv = (x + size[0]) / dx - j, (y + size[1]) / dy - i
    V = lambda a, b: np.array([-size[0] + b * dx, -size[1] + a * dy, size[2] * elev[a, b]])
    tri = [V(i, j), V(i, j + 1), V(i + 1, j + 1)] if fu >= fv else [V(i, j), V(i + 1, j + 1), V(i + 1, j)]
    A = np.array([[t[0], t[1], 1.0] for t in tri]).T
    w = np.linalg.solve(A, [x, y, 1.0])
    hgt = w @ np.array([t[2] for t in tri])
    nt = np.cross(tri[1] - tri[0], tri[2] - tri[0]); nt /= np.linalg.norm(nt)
    tip = np.array([x, y, hgt - 0.01])
    verts = np.array([[0, 0, -0.05], [0.04, 0, 0.02], [-0.02, 0.035, 0.02], [-0.02, -0.035, 0.02]])
    face = [(0, 2, 1), (0, 3, 2), (0, 1, 3), (1, 2, 3)]
    I3 = np.eye(3).ravel()
    got = O.collide_mesh(I3, np.zeros(3), I3, tip - verts[0], verts, face, size=size, elev=elev)
    k = np.argmin(got[:, 0])
    assert got[k, 0] == pytest.approx(nt[2] * (tip[2] - hgt), abs=1e-12)
    np.testing.assert_allclose(got[k, 4:7], nt, atol=1e-12)


def test_hull_comes_to_rest_on_the_plane_carrying_its_weight():
    """a seeded hull dropped on a frictional plane: settled (its height no longer changes; the soft
    pyramidal contacts leave a slow creep, as for the cylinder's tripod) its contacts' normal
    forces sum to m g"""
    m = W.hulls()
    om = O.OracleModel(m)
    q0 = m.qpos_init.astype(np.float64)[None]
    v0 = np.zeros((1, m.nv))
    q, v, _, _ = om.rollout(q0, v0, np.zeros((1500, 1, 0)), 1, solver_cap=-1)
    assert abs(v[0, 2]) < 1e-5 and np.abs(v[0, :6]).max() < 5e-3
    f = om.forward(q[0], v[0], np.zeros(m.nv), None, solver_cap=-1)
    rows, con = f["rows"][: f["nrow"]], f["contacts"]
    # the first hull's pair is pair 0: its slots 0..3; pyramid edges carry normal force sum(f_e)
    act = np.where(con[:4, 0] > 0)[0]
    fn = rows[: 4 * len(act), m.nv + 6].sum()
    assert fn == pytest.approx(0.3 * 9.81, rel=1e-3)
