"""Pins of the oracle's collision functions that share nothing with how the oracle computes them:

* box-box face manifolds against exact vertex enumeration of the contact polygon (the pairwise
  intersections of its eight bounding lines in the incident face's plane, kept where feasible);
* capsule-box (R15: the capsule's two end spheres against the box) against a dense sampling of
  the box surface, and, where a capsule enters the box end first, against the sampled
  support-function penetration depth;
* sphere-capsule against a dense search over the segment parameter;
* the contact frame (R14) against frames worked out by hand.

Each docstring names the mistakes the pin catches."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_08844_b300 import workloads as W


def rot_z(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])


def rot_axis(axis, a):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(a) * K + (1 - np.cos(a)) * K @ K


def polygon_vertices(lines):
    """Vertices of {x in R^2: g . x <= c for every (g, c)}: every pairwise intersection of the
    boundary lines that satisfies all constraints (duplicates merged)."""
    out = []
    for (g1, c1), (g2, c2) in itertools.combinations(lines, 2):
        A = np.array([g1, g2])
        if abs(np.linalg.det(A)) < 1e-14:
            continue
        x = np.linalg.solve(A, [c1, c2])
        if all(g @ x <= c + 1e-12 for g, c in lines) and not any(np.abs(x - y).max() < 1e-10 for y in out):
            out.append(x)
    return out


def face_manifold(pr, Rr, hr, kr, sr, fc, iu, iv, hu, hv):
    """Exact contact polygon of an incident face (centre fc, unit axes iu, iv, half-extents hu, hv)
    against the reference face of box (pr, Rr, hr) with outward normal sr * Rr[:, kr]: the face's
    points inside the reference face's prism, enumerated from the eight bounding lines in the face's
    coordinates (a, b); returns [(vertex, depth below the reference face)] for depth >= 0."""
    o = [k for k in range(3) if k != kr]
    lines = [(np.array([1.0, 0]), hu), (np.array([-1.0, 0]), hu), (np.array([0, 1.0]), hv), (np.array([0, -1.0]), hv)]
    for k in o:   # |(p - pr) . e_k| <= hr_k, linear in (a, b)
        e = Rr[:, k]
        g = np.array([iu @ e, iv @ e])
        c0 = (fc - pr) @ e
        lines += [(g, hr[k] - c0), (-g, hr[k] + c0)]
    nref = sr * Rr[:, kr]
    out = []
    for a, b in polygon_vertices(lines):
        p = fc + a * iu + b * iv
        d = hr[kr] - (p - pr) @ nref
        if d >= 0:
            out.append((p, d))
    return out


def test_box_box_face_manifold_matches_vertex_enumeration():
    """Box B lies tilted on box A's top face (random yaw, up to 3 degrees of tilt, random offset so
    that the faces overlap partly, 1-8 mm of penetration).  The contact normal is then A's +z
    (reference face A's top, incident face B's bottom) or B's -z (reference face B's bottom,
    incident face A's top).  The manifold is the part of the incident face inside the reference
    face's prism: enumerated exactly from its eight bounding lines, the vertices below the
    reference face are the contacts when at most four; with more, the four kept are among them and
    the first kept is the deepest.  A missing or wrong side plane, a wrong incident face, a dropped
    prism-edge vertex, a wrong depth sign or swapped roles of the boxes fails here."""
    r = np.random.default_rng(41)
    cases = {"A": 0, "B": 0}
    reduced = 0
    for trial in range(500):
        hA = r.uniform(0.05, 0.3, 3)
        hB = r.uniform(0.05, 0.3, 3)
        RB = rot_z(r.uniform(0, 2 * np.pi)) @ rot_axis(r.normal(size=3) * [1, 1, 0] + [0, 0, 1e-9],
                                                        np.radians(r.uniform(0, 3)))
        corners = [RB @ np.array([sx * hB[0], sy * hB[1], -hB[2]]) for sx in (-1, 1) for sy in (-1, 1)]
        low = min(c[2] for c in corners)
        xy = r.uniform(-1, 1, 2) * (hA[:2] + 0.5 * hB[:2])
        pB = np.array([xy[0], xy[1], hA[2] - low - r.uniform(0.001, 0.008)])
        out = O.collide(W.BOX, np.eye(3), np.zeros(3), hA, W.BOX, RB, pB, hB)
        act = out[out[:, 0] < 1]
        if len(act) == 0:
            continue
        n = act[0, 4:7]
        if np.abs(n - [0, 0, 1]).max() <= 1e-12:      # reference: A's top face
            ref = "A"
            below = face_manifold(np.zeros(3), np.eye(3), hA, 2, 1.0, pB - RB[:, 2] * hB[2], RB[:, 0], RB[:, 1],
                                  hB[0], hB[1])
            nref = n
        elif np.abs(n + RB[:, 2] * -1).max() <= 1e-12:   # reference: B's bottom face (normal A -> B = B's +z)
            ref = "B"
            below = face_manifold(pB, RB, hB, 2, -1.0, np.array([0, 0, hA[2]]), np.array([1.0, 0, 0]),
                                  np.array([0, 1.0, 0]), hA[0], hA[1])
            nref = -n
        else:
            continue   # an edge or side axis won: not this pin's case
        got = [row[1:4] - nref * (-row[0]) / 2 for row in act]   # midpoint -> the polygon vertex
        depths = -act[:, 0]
        assert len(below) > 0
        if len(below) <= 4:
            assert len(got) == len(below), (trial, ref, len(got), len(below))
        else:
            reduced += 1
            assert len(got) == 4
            assert depths[0] == pytest.approx(max(d for _, d in below), abs=1e-12)
        for g, dep in zip(got, depths):
            j = int(np.argmin([np.abs(g - p).max() for p, _ in below]))
            assert np.abs(g - below[j][0]).max() < 1e-9, (trial, ref)
            assert dep == pytest.approx(below[j][1], abs=1e-12)
        cases[ref] += 1
    assert cases["A"] >= 40 and cases["B"] >= 40 and reduced >= 5, (cases, reduced)


def box_signed_distance(p, R, c, h, n=81):
    """Signed distance from p to the box (frame R, centre c, half-sizes h): the distance to the
    nearest of a dense grid of surface points, refined on a finer grid around it, negative inside."""
    q = R.T @ (p - c)
    inside = np.all(np.abs(q) <= h)
    best, best_pt = np.inf, None
    for axis in range(3):
        for sgn in (-1, 1):
            o = [k for k in range(3) if k != axis]
            lo = np.array([-h[o[0]], -h[o[1]]]); hi = -lo
            for it in range(4):
                u = np.linspace(lo[0], hi[0], n); v = np.linspace(lo[1], hi[1], n)
                U, V = np.meshgrid(u, v)
                pts = np.zeros(U.shape + (3,))
                pts[..., axis] = sgn * h[axis]; pts[..., o[0]] = U; pts[..., o[1]] = V
                d = np.linalg.norm(pts - q, axis=-1)
                i = np.unravel_index(np.argmin(d), d.shape)
                if d[i] < best:
                    best, best_pt = d[i], pts[i]
                step = np.array([(hi[0] - lo[0]) / (n - 1), (hi[1] - lo[1]) / (n - 1)])
                ctr = np.array([U[i], V[i]])
                lo = np.maximum(ctr - 2 * step, [-h[o[0]], -h[o[1]]]); hi = np.minimum(ctr + 2 * step, [h[o[0]], h[o[1]]])
    return (-best if inside else best), R @ best_pt + c


def test_capsule_box_end_spheres_match_sampled_surface_distance():
    """Capsule (geom1) against box (geom2): each contact is one end sphere's signed distance to the
    box minus the radius (R15), measured here against the box surface sampled densely.  A contact
    taken at the capsule's centre, a dropped radius or an inside point measured to the wrong face
    fails here."""
    r = np.random.default_rng(7)
    for trial in range(40):
        h = r.uniform(0.03, 0.1, 3)
        R = rot_axis(r.normal(size=3), r.uniform(0, np.pi))
        rad, half = r.uniform(0.005, 0.02), r.uniform(0.01, 0.05)
        Rc = rot_axis(r.normal(size=3), r.uniform(0, np.pi))
        a = Rc[:, 2]
        pc = r.normal(size=3) * 0.05
        out = O.collide(W.CAPSULE, Rc, pc, [rad, half], W.BOX, R, np.zeros(3), h)
        assert out.shape[0] == 2
        for k, s in enumerate((-half, half)):
            sd, _ = box_signed_distance(pc + s * a, R, np.zeros(3), h)
            assert out[k, 0] == pytest.approx(sd - rad, abs=2e-6), (trial, k)


def test_capsule_entering_box_end_first_matches_support_penetration():
    """A capsule entering a box end first, axis within 20 degrees of the face normal: its deepest
    point is the entering end's sphere, so the deepest contact is the capsule-box penetration depth,
    the minimum over directions u of s_capsule(u) + s_box(-u) (support functions), sampled.  The
    end-sphere reading at the wrong end, or a sign error in the depth, fails here."""
    r = np.random.default_rng(8)
    dirs = r.normal(size=(200000, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    for trial in range(12):
        h = r.uniform(0.04, 0.1, 3)
        rad, half = 0.01, 0.04
        Rc = rot_axis(r.normal(size=3) * [1, 1, 0] + [0, 0, 1e-9], np.radians(r.uniform(0, 20)))
        a = Rc[:, 2]
        pen = r.uniform(0.001, 0.01)
        xy = r.uniform(-0.5, 0.5, 2) * h[:2]
        low_end = np.array([xy[0], xy[1], 0.0]) - a * half        # the lower end's centre before the shift
        pc = np.array([xy[0], xy[1], 0.0]) + np.array([0, 0, h[2] + rad - pen - low_end[2]])
        out = O.collide(W.CAPSULE, Rc, pc, [rad, half], W.BOX, np.eye(3), np.zeros(3), h)
        f = lambda D: D @ pc + half * np.abs(D @ a) + rad + np.abs(D) @ h   # s_capsule(u) + s_box(-u)
        vals = f(dirs)
        best, depth = dirs[np.argmin(vals)], vals.min()
        gen, step = np.random.default_rng(0), 0.05
        for _ in range(60):   # shrinking random local search around the sampled minimum
            cand = best + step * gen.normal(size=(2000, 3))
            cand /= np.linalg.norm(cand, axis=1, keepdims=True)
            fc = f(cand)
            if fc.min() < depth:
                depth, best = fc.min(), cand[np.argmin(fc)]
            step *= 0.8
        assert -out[:, 0].min() == pytest.approx(depth, abs=2e-5)
        assert -out[:, 0].min() == pytest.approx(pen, abs=1e-9)


def test_sphere_capsule_matches_segment_search():
    """Sphere (geom1) against capsule (geom2): distance to the segment's nearest point (a dense
    search over the segment parameter, then a finer one) minus both radii, the normal from the
    sphere towards that point, the contact midway between the two surface points.  Clamping to
    the wrong end, or a normal pointing from the capsule to the sphere, fails here."""
    r = np.random.default_rng(9)
    for trial in range(40):
        c1 = r.normal(size=3) * 0.1
        r1, r2, half = r.uniform(0.01, 0.05), r.uniform(0.01, 0.05), r.uniform(0.02, 0.2)
        R2 = rot_axis(r.normal(size=3), r.uniform(0, np.pi))
        c2 = r.normal(size=3) * 0.1
        a = R2[:, 2]
        out = O.collide(W.SPHERE, np.eye(3), c1, [r1], W.CAPSULE, R2, c2, [r2, half])
        s = np.linspace(-half, half, 20001)
        d = np.linalg.norm(c2 + s[:, None] * a - c1, axis=1)
        i = np.argmin(d)
        lo, hi = s[max(i - 1, 0)], s[min(i + 1, len(s) - 1)]
        s = np.linspace(lo, hi, 20001)
        d = np.linalg.norm(c2 + s[:, None] * a - c1, axis=1)
        i = np.argmin(d)
        q = c2 + s[i] * a
        n = (q - c1) / np.linalg.norm(q - c1)
        assert out[0, 0] == pytest.approx(d[i] - r1 - r2, abs=1e-9)
        assert np.abs(out[0, 4:7] - n).max() < 1e-6
        mid = 0.5 * ((c1 + r1 * n) + (q - r2 * n))
        assert np.abs(out[0, 1:4] - mid).max() < 1e-6


@pytest.mark.parametrize("n,t1,t2", [
    ((0, 0, 1), (0, 1, 0), (-1, 0, 0)),        # |n_x| = |n_y| = 0: the tie goes to x
    ((1, 0, 0), (0, 0, 1), (0, -1, 0)),        # tie between y and z: y
    ((0, 1, 0), (0, 0, -1), (-1, 0, 0)),       # tie between x and z: x
    ((0, 0, -1), (0, -1, 0), (-1, 0, 0)),      # a downward normal
])
def test_contact_frame_by_hand(n, t1, t2):
    """R14: t1 = normalise(n x e_k), e_k the world axis of smallest |n_k| (ties to the lowest k),
    t2 = n x t1; the frames above are worked out by hand.  Choosing the largest |n_k| (n x e_k = 0
    for an axis-aligned normal), the highest k on ties, or t2 = t1 x n fails here."""
    n = np.array(n, float)
    R = np.eye(3)
    R[:, 2] = n   # a plane whose normal is n (its other axes do not enter the frame)
    out = O.collide(W.PLANE, R, np.zeros(3), [0, 0, 0], W.SPHERE, np.eye(3), n * 0.05, [0.1])
    assert np.allclose(out[0, 4:7], n, atol=1e-12)
    assert np.allclose(out[0, 7:10], t1, atol=1e-12)
    assert np.allclose(out[0, 10:13], t2, atol=1e-12)


def test_contact_frame_general_normal_by_hand():
    """n = (1, 1, 0.5) / 1.5: smallest |n_k| is z, so t1 = normalise(n x e_z) = (1, -1, 0) / sqrt 2
    and t2 = n x t1 = (1, 1, -4) / (3 sqrt 2)."""
    n = np.array([1.0, 1.0, 0.5]) / 1.5
    R = np.eye(3)
    R[:, 2] = n
    out = O.collide(W.PLANE, R, np.zeros(3), [0, 0, 0], W.SPHERE, np.eye(3), n * 0.05, [0.1])
    assert np.allclose(out[0, 7:10], np.array([1.0, -1.0, 0.0]) / np.sqrt(2), atol=1e-12)
    assert np.allclose(out[0, 10:13], np.array([1.0, 1.0, -4.0]) / (3 * np.sqrt(2)), atol=1e-12)
