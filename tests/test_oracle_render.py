"""Pins of the oracle's ray tracer (oracle/render.py) against closed-form silhouettes, horizons
and shadows, and against ray marching through the shapes' inside tests."""
import dataclasses
import math

import numpy as np
import pytest

from paper_2502_08844_b300 import workloads as W
from oracle import oracle as O
from oracle import render as RD


def _scene(**kw):
    base = dict(cam_pos=(0.0, 0.0, 0.0), cam_lookat=(1.0, 0.0, 0.0), cam_up=(0.0, 0.0, 1.0), fovy_deg=40.0,
                width=41, height=31, light_dir=(0.0, 0.0, -1.0), ambient=0.25, diffuse=0.75,
                background=(0.1, 0.2, 0.3), geom_rgb=np.array([[1.0, 1.0, 1.0]], np.float32))
    base.update(kw)
    return W.Scene(**base)


def _one_geom_model(gtype, size, pos=(0, 0, 0), quat=(1, 0, 0, 0)):
    b = W.ModelBuilder("one")
    b.geom(0, gtype, size, pos=pos, quat=quat)
    return b.build(timestep=0.01)


def test_centre_ray_is_the_view_direction():
    cam, D = RD.camera_rays(_scene())
    assert np.allclose(cam, 0) and np.allclose(D[15, 20], [1, 0, 0], atol=1e-15)


def test_sphere_silhouette_and_centre_shade():
    """A ray hits a sphere (centre c at distance L, radius r) iff its angle to c is below
    asin(r / L); the centre pixel sees the normal -d."""
    c, r = np.array([3.0, 0.0, 0.0]), 0.6
    m = _one_geom_model(W.SPHERE, (r,), pos=c)
    sc = _scene(light_dir=(1.0, 0.0, 0.0))
    col, code = RD.render(O.OracleModel(m), sc, np.zeros(0))
    _, D = RD.camera_rays(sc)
    ang = np.arccos(np.clip(D @ (c / np.linalg.norm(c)), -1, 1))
    margin = np.abs(ang - math.asin(r / 3.0))
    expect = ang < math.asin(r / 3.0)
    assert np.array_equal((code > 0)[margin > 1e-9], expect[margin > 1e-9])
    assert expect.sum() > 30
    # light travelling along +x (from behind the camera) meets the camera-facing side head on
    assert np.allclose(col[15, 20], 1.0)
    sc2 = _scene(light_dir=(-1.0, 0.0, 0.0))          # from behind the sphere: ambient only
    col2, _ = RD.render(O.OracleModel(m), sc2, np.zeros(0))
    assert np.allclose(col2[15, 20], 0.25)


def test_plane_horizon_and_constant_shade():
    """Camera 1 m above the floor looking along +x: rays pointing down hit the floor, others
    miss; an unshadowed floor is shaded ambient + diffuse (n . l = 1 with light straight down)."""
    m = _one_geom_model(W.PLANE, (0, 0, 0), pos=(0, 0, -1.0))
    col, code = RD.render(O.OracleModel(m), _scene(), np.zeros(0))
    _, D = RD.camera_rays(_scene())
    down = D[..., 2] < 0
    assert np.array_equal(code > 0, down)
    assert np.allclose(col[down], 1.0) and np.allclose(col[~down], [0.1, 0.2, 0.3])


def test_plane_seen_from_below():
    m = _one_geom_model(W.PLANE, (0, 0, 0), pos=(0, 0, 1.0))
    col, code = RD.render(O.OracleModel(m), _scene(light_dir=(0.0, 0.0, 1.0)), np.zeros(0))
    _, D = RD.camera_rays(_scene())
    up = D[..., 2] > 0
    assert np.array_equal(code > 0, up) and np.allclose(col[up], 1.0)   # the lower face, lit from below


def test_sphere_shadow_on_the_floor():
    """Light straight down: the floor point under a sphere's centre is in shadow, a point 1 m
    away is lit."""
    b = W.ModelBuilder("shadow")
    b.geom(0, W.PLANE, (0, 0, 0))
    b.geom(0, W.SPHERE, (0.3,), pos=(3.0, 0.0, 0.6))
    m = b.build(timestep=0.01)
    sc = _scene(cam_pos=(0.0, 0.0, 2.0), cam_lookat=(3.0, 0.0, 0.0), width=81, height=61,
                geom_rgb=np.array([[0.5, 0.5, 0.5], [1, 0, 0]], np.float32))
    col, code = RD.render(O.OracleModel(m), sc, np.zeros(0))
    cam, D = RD.camera_rays(sc)

    def pixel_of(p):
        v = p - cam
        k = np.argmax((D / np.linalg.norm(D, axis=-1, keepdims=True)) @ (v / np.linalg.norm(v)))
        return np.unravel_index(k, D.shape[:2])

    under = pixel_of(np.array([3.0, 0.0, 0.0]))
    if code[under] == 1 + 65536:                       # visible floor point, in shadow
        assert np.allclose(col[under], 0.5 * 0.25)
    else:
        assert code[under] == 2                        # or hidden behind the sphere itself
    lit = pixel_of(np.array([3.0, 1.2, 0.0]))
    assert code[lit] == 1 and np.allclose(col[lit], 0.5 * 1.0)
    assert np.any(code == 1 + 65536)


def _march(inside, O_, d, tmax=10.0, step=2e-5):
    ts = np.arange(0.0, tmax, step)
    pts = O_[None, :] + ts[:, None] * d[None, :]
    k = np.argmax(inside(pts))
    return ts[k] if inside(pts[k:k + 1])[0] else np.inf


@pytest.mark.parametrize("gtype", [W.BOX, W.CAPSULE, W.CYLINDER])
def test_box_capsule_and_cylinder_hits_match_ray_marching(gtype):
    rng = np.random.default_rng(7 + gtype)
    q = np.array([0.9, 0.2, -0.3, 0.25]); q /= np.linalg.norm(q)
    x = np.array([2.0, 0.1, -0.2])
    size = (0.3, 0.2, 0.15) if gtype == W.BOX else ((0.15, 0.35) if gtype == W.CAPSULE else (0.2, 0.25))
    m = _one_geom_model(gtype, size, pos=x, quat=q)
    om = O.OracleModel(m)
    Rg, Xg = om.geom_frames(np.zeros(0))
    R, X = Rg[0], Xg[0]
    if gtype == W.BOX:
        inside = lambda P: np.all(np.abs((P - X) @ R) <= np.array(size), axis=1)
    elif gtype == W.CYLINDER:
        def inside(P):
            L = (P - X) @ R
            return (np.hypot(L[:, 0], L[:, 1]) <= size[0]) & (np.abs(L[:, 2]) <= size[1])
    else:
        def inside(P):
            L = (P - X) @ R
            z = np.clip(L[:, 2], -size[1], size[1])
            return np.hypot(L[:, 0], L[:, 1]) ** 2 + (L[:, 2] - z) ** 2 <= size[0] ** 2
    hits = 0
    for _ in range(40):
        O_ = np.array([0.0, 0.0, 0.0]) + rng.normal(0, 0.05, 3)
        d = (X - O_) + rng.normal(0, 0.25, 3)
        d /= np.linalg.norm(d)
        t, n = RD.intersect(gtype, X, R, np.array(size, np.float64), O_, d[None, :])
        tm = _march(inside, O_, d)
        if np.isfinite(tm):
            hits += 1
            assert t[0] == pytest.approx(tm, abs=3e-5)
            # the normal is outward: a small step along it leaves the shape
            assert not inside((O_ + d * t[0] + n[0] * 1e-4)[None, :])[0]
        else:
            assert not np.isfinite(t[0]) or t[0] == pytest.approx(tm, abs=3e-5)
    assert hits >= 10
