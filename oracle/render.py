"""FP64 oracle of the batch ray tracer (pg_render) -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg import this
module.  It draws what the library's pixel observations draw (the paper renders pixel
observations with a CUDA batch ray tracer, Sec. 5): a pinhole camera, every drawn geom at the
pose the oracle's own forward kinematics gives, the nearest hit per ray (first geom on ties),
Lambertian shading under one directional light with an ambient term, and hard shadows from one
shadow ray per hit.  A point is lit when its surface faces the light and no drawn geom blocks
its shadow ray (the shadow ray here tests every drawn geom, the one hit included).  Written with numpy over all pixels of one image at a time.

Readings where the paper leaves the choice: pixel (x, y) has y = 0 at the top and its ray goes
through the pixel's centre; planes are infinite and seen from both faces; a shadow ray starts
1e-4 off the surface along its normal and any drawn geom in front of it blocks the light;
hits closer than 1e-5 are ignored; colours are quantised as round(255 * clip(c, 0, 1)).
"""
from __future__ import annotations

import numpy as np

EPS_T = 1e-5
LIFT = 1e-4
PLANE, SPHERE, CAPSULE, BOX, CYLINDER = 0, 1, 2, 3, 5


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def camera_rays(scene):
    """Origin (3,) and unit directions [H, W, 3] of the primary rays."""
    W_, H_ = int(scene.width), int(scene.height)
    pos = np.asarray(scene.cam_pos, np.float64)
    f = _unit(np.asarray(scene.cam_lookat, np.float64) - pos)
    r = _unit(np.cross(f, np.asarray(scene.cam_up, np.float64)))
    u = np.cross(r, f)
    th = np.tan(np.radians(float(np.float32(scene.fovy_deg))) / 2)
    sx = 2 * (np.arange(W_) + 0.5) / W_ - 1
    sy = 1 - 2 * (np.arange(H_) + 0.5) / H_
    d = f[None, None, :] + (sx[None, :, None] * th * W_ / H_) * r + (sy[:, None, None] * th) * u
    return pos, d / np.linalg.norm(d, axis=-1, keepdims=True)


def _sphere(O, D, c, r):
    oc = O - c
    b = np.sum(oc * D, -1)
    cc = np.sum(oc * oc, -1) - r * r
    disc = b * b - cc
    sq = np.sqrt(np.maximum(disc, 0))
    t = -b - sq
    t = np.where(t > EPS_T, t, -b + sq)
    ok = (disc >= 0) & (t > EPS_T)
    n = (O + D * np.where(ok, t, 0.0)[..., None] - c) / r
    return np.where(ok, t, np.inf), n


def intersect(gtype, x, R, size, O, D):
    """Nearest hit distance beyond EPS_T (inf on a miss) and the surface normal facing the ray
    (outward for closed shapes), for rays O + t D ([P, 3] or (3,) origins, [P, 3] directions)."""
    O = np.broadcast_to(np.asarray(O, np.float64), D.shape)
    if gtype == PLANE:
        nz = R[:, 2]
        den = D @ nz
        with np.errstate(divide="ignore", invalid="ignore"):
            t = ((x - O) @ nz) / den
        ok = (np.abs(den) >= 1e-12) & (t > EPS_T)
        n = np.where((den < 0)[:, None], nz, -nz)
        return np.where(ok, t, np.inf), n
    if gtype == SPHERE:
        return _sphere(O, D, x, size[0])
    lo = (O - x) @ R            # R^T (O - x), row-wise
    ld = D @ R
    if gtype == CAPSULE:
        r, h = size[0], size[1]
        best = np.full(D.shape[0], np.inf)
        nl = np.zeros_like(D)
        a = ld[:, 0] ** 2 + ld[:, 1] ** 2
        b = lo[:, 0] * ld[:, 0] + lo[:, 1] * ld[:, 1]
        c = lo[:, 0] ** 2 + lo[:, 1] ** 2 - r * r
        disc = b * b - a * c
        good = (a > 1e-12) & (disc >= 0)
        sq = np.sqrt(np.maximum(disc, 0))
        for sgn in (-1.0, 1.0):
            with np.errstate(divide="ignore", invalid="ignore"):
                t = (-b + sgn * sq) / a
            z = lo[:, 2] + t * ld[:, 2]
            take = good & (t > EPS_T) & (t < best) & (np.abs(z) <= h)
            best = np.where(take, t, best)
            p = lo + ld * t[:, None]
            nl = np.where(take[:, None], np.stack([p[:, 0] / r, p[:, 1] / r, np.zeros_like(t)], -1), nl)
        for zc in (-h, h):
            t, ns = _sphere(lo, ld, np.array([0.0, 0.0, zc]), r)
            take = t < best
            best = np.where(take, t, best)
            nl = np.where(take[:, None], ns, nl)
        return best, nl @ R.T
    if gtype == CYLINDER:
        r, h = size[0], size[1]
        best = np.full(D.shape[0], np.inf)
        nl = np.zeros_like(D)
        a = ld[:, 0] ** 2 + ld[:, 1] ** 2
        b = lo[:, 0] * ld[:, 0] + lo[:, 1] * ld[:, 1]
        c = lo[:, 0] ** 2 + lo[:, 1] ** 2 - r * r
        disc = b * b - a * c
        good = (a > 1e-12) & (disc >= 0)
        sq = np.sqrt(np.maximum(disc, 0))
        for sgn in (-1.0, 1.0):            # the side, within the caps
            with np.errstate(divide="ignore", invalid="ignore"):
                t = (-b + sgn * sq) / a
            z = lo[:, 2] + t * ld[:, 2]
            take = good & (t > EPS_T) & (t < best) & (np.abs(z) <= h)
            best = np.where(take, t, best)
            p = lo + ld * t[:, None]
            nl = np.where(take[:, None], np.stack([p[:, 0] / r, p[:, 1] / r, np.zeros_like(t)], -1), nl)
        for zc in (-h, h):                 # the two cap discs
            with np.errstate(divide="ignore", invalid="ignore"):
                t = (zc - lo[:, 2]) / ld[:, 2]
            p = lo + ld * np.where(np.isfinite(t), t, 0.0)[:, None]
            take = (np.abs(ld[:, 2]) > 1e-12) & (t > EPS_T) & (t < best) & (p[:, 0] ** 2 + p[:, 1] ** 2 <= r * r)
            best = np.where(take, t, best)
            nl = np.where(take[:, None], np.array([0.0, 0.0, 1.0 if zc > 0 else -1.0]), nl)
        return best, nl @ R.T
    # box: slabs in the box frame
    hs = np.asarray(size, np.float64)
    tn = np.full(D.shape[0], -np.inf); tf = np.full(D.shape[0], np.inf)
    an = np.zeros(D.shape[0], int); af = np.zeros(D.shape[0], int)
    sn = np.ones(D.shape[0]); sf = np.ones(D.shape[0])
    miss = np.zeros(D.shape[0], bool)
    for k in range(3):
        par = np.abs(ld[:, k]) < 1e-12
        miss |= par & (np.abs(lo[:, k]) > hs[k])
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (-hs[k] - lo[:, k]) / ld[:, k]
            t2 = (hs[k] - lo[:, k]) / ld[:, k]
        swap = t1 > t2
        lo_t, hi_t = np.where(swap, t2, t1), np.where(swap, t1, t2)
        s_lo, s_hi = np.where(swap, 1.0, -1.0), np.where(swap, -1.0, 1.0)
        upd = ~par & (lo_t > tn)
        tn = np.where(upd, lo_t, tn); an = np.where(upd, k, an); sn = np.where(upd, s_lo, sn)
        upd = ~par & (hi_t < tf)
        tf = np.where(upd, hi_t, tf); af = np.where(upd, k, af); sf = np.where(upd, s_hi, sf)
    inside = ~(tn > EPS_T)
    t = np.where(inside, tf, tn)
    ok = ~miss & ~(tn > tf) & (tf > EPS_T)
    ax = np.where(inside, af, an)
    sg = np.where(inside, sf, sn)
    nl = np.zeros_like(D)
    nl[np.arange(D.shape[0]), ax] = sg
    return np.where(ok, t, np.inf), nl @ R.T


def randomized_scene(scene, cam_offset=None, light_dir=None):
    """The scene one environment sees under visual randomisation: the camera moved by cam_offset
    (its look-at point kept), the light along light_dir."""
    import dataclasses
    kw = {}
    if cam_offset is not None:
        kw["cam_pos"] = tuple(np.asarray(scene.cam_pos, np.float64) + np.asarray(cam_offset, np.float64))
    if light_dir is not None:
        kw["light_dir"] = tuple(np.asarray(light_dir, np.float64))
    return dataclasses.replace(scene, **kw)


def render(om, scene, qpos):
    """One image of one environment: colours [H, W, 3] (float) and hit codes [H, W] (0
    background, geom + 1, plus 65536 when no direct light reaches the point)."""
    Rg, Xg = om.geom_frames(np.asarray(qpos, np.float64))
    m = om.src
    rgb = np.asarray(scene.geom_rgb, np.float64)
    drawn = [g for g in range(m.ngeom) if rgb[g, 0] >= 0 and m.geom_type[g] in (PLANE, SPHERE, CAPSULE, BOX, CYLINDER)]
    cam, D = camera_rays(scene)
    H_, W_ = D.shape[:2]
    D = D.reshape(-1, 3)
    size = m.geom_size.astype(np.float64)
    best = np.full(D.shape[0], np.inf)
    hit = np.full(D.shape[0], -1)
    nrm = np.zeros_like(D)
    for g in drawn:
        t, n = intersect(int(m.geom_type[g]), Xg[g], Rg[g], size[g], cam, D)
        take = t < best
        best = np.where(take, t, best); hit = np.where(take, g, hit); nrm = np.where(take[:, None], n, nrm)
    light = -_unit(np.asarray(scene.light_dir, np.float64))
    any_hit = hit >= 0
    Q = cam + D * np.where(any_hit, best, 0)[:, None] + nrm * LIFT
    Ld = np.broadcast_to(light, D.shape)
    blocked = np.zeros(D.shape[0], bool)
    for g in drawn:
        t, _ = intersect(int(m.geom_type[g]), Xg[g], Rg[g], size[g], Q, Ld)
        blocked |= np.isfinite(t)
    nl = nrm @ light
    lit = any_hit & (nl > 0) & ~blocked          # facing the light and not blocked
    shade = float(np.float32(scene.ambient)) + np.where(lit, float(np.float32(scene.diffuse)) * nl, 0)
    col = np.where(any_hit[:, None], rgb[np.maximum(hit, 0)] * shade[:, None], np.asarray(scene.background, np.float64))
    code = np.where(any_hit, hit + 1 + np.where(lit, 0, 65536), 0)
    return col.reshape(H_, W_, 3), code.reshape(H_, W_)


def quantise(col):
    return np.clip(np.rint(255 * col), 0, 255).astype(np.uint8)
