"""GPU parity of the batch ray tracer (pg_render) against the FP64 oracle (oracle/render.py)
through the C ABI.

Which geom a ray hits, and whether its hit point is in shadow, are decided by floating-point
comparisons; along a silhouette or a shadow edge a float32 ray and a float64 ray can go either
way, and both images are then correct.  So the hit codes must agree on every pixel except
those on an edge of the oracle's own code map (a 4-neighbour with another code), and at most
1 % of the pixels may differ at all.  Where the codes agree off an edge, float colours agree to
1e-4 (the rounding of a dot product of unit vectors and a few products) and uint8 colours to one
code.  On an edge of a round shape the hit distance is the square root of a vanishing
discriminant, so the shading normal's error grows like the square root of the rounding (~3e-4
at float32): there agreeing pixels are held to 2e-2."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import render as RD
from paper_2502_08844_b300 import core, workloads as W
from tests.gpu_helpers import GpuRun

pytestmark = pytest.mark.gpu


def _edge(code):
    e = np.zeros_like(code, bool)
    e[1:, :] |= code[1:, :] != code[:-1, :]
    e[:-1, :] |= code[:-1, :] != code[1:, :]
    e[:, 1:] |= code[:, 1:] != code[:, :-1]
    e[:, :-1] |= code[:, :-1] != code[:, 1:]
    return e


def _render_gpu(run, scene, fmt):
    n = run.n
    px = torch.zeros((n, scene.height, scene.width, 3), dtype=torch.uint8 if fmt == "u8" else torch.float32,
                     device="cuda")
    hits = torch.zeros((n, scene.height, scene.width), dtype=torch.int32, device="cuda")
    core.render(run.batch, run.state, scene, px, hits)
    torch.cuda.synchronize()
    return px.cpu().numpy(), hits.cpu().numpy()


def _check(m, scene, q, v, n):
    om = O.OracleModel(m)
    run = GpuRun(m, n)
    run.set_state(q, v)
    colf, hits = _render_gpu(run, scene, "f32")
    col8, hits8 = _render_gpu(run, scene, "u8")
    assert np.array_equal(hits, hits8)
    differ = 0
    drawn = 0
    for e in range(n):
        oc, ocode = RD.render(om, scene, q[e].astype(np.float64))
        bad = hits[e] != ocode
        assert not np.any(bad & ~_edge(ocode)), e
        differ += bad.sum()
        edge = _edge(ocode)
        same = ~bad & ~edge
        assert np.abs(colf[e][same] - oc[same]).max() <= 1e-4, e
        assert np.abs(col8[e][same].astype(int) - RD.quantise(oc)[same].astype(int)).max() <= 1, e
        on_edge = ~bad & edge
        if on_edge.any():
            assert np.abs(colf[e][on_edge] - oc[on_edge]).max() <= 2e-2, e
        drawn += (ocode > 0).sum()
    assert differ <= 0.01 * n * scene.width * scene.height
    return drawn


def test_cartpole_pixels_match_oracle():
    m = W.cartpole_pixels()
    n = 48
    q, v = W.initial_state(m, 0, n)
    q = q.copy(); q[:, 0] *= 8.0; q[:, 1] *= 12.0          # carts across the view, poles swinging
    drawn = _check(m, W.cartpole_scene(), q, v, n)
    assert drawn > n * 1000


def test_quadruped_pixels_match_oracle():
    m = W.quadruped()
    om = O.OracleModel(m)
    q0, v0 = W.initial_state(m, 1, 12)
    U = W.actions(m, 1, 12, 0, 40)
    q, v, _, _ = om.rollout(q0, v0, U, 5)          # varied poses after 40 control steps
    drawn = _check(m, W.quadruped_scene(48, 40), q.astype(np.float32), v.astype(np.float32), 12)
    assert drawn > 12 * 500


def test_cylinder_pixels_match_oracle():
    """Cylinders (side and cap discs) on a plane, in the poses of the contact tests: falling tilted,
    rolling on the side, standing on a cap."""
    from tests.test_gpu_cylinder import _cylinder_scene, _initial_states
    m = _cylinder_scene()
    om = O.OracleModel(m)
    q0, v0 = _initial_states()
    q0 = np.repeat(q0, 4, 0)
    v0 = np.repeat(v0, 4, 0)
    q0[:, 0] = np.tile([0.0, 0.02, -0.02, 0.04], 3)          # all in view
    q0[:, 1] = 0.0
    q, v, _, _ = om.rollout(q0, v0, np.zeros((30, 12, 0)), 4)
    scene = W.Scene(cam_pos=(0.3, -0.3, 0.22), cam_lookat=(0.03, 0.0, 0.07), cam_up=(0.0, 0.0, 1.0), fovy_deg=50.0,
                    width=48, height=40, light_dir=(-0.3, 0.4, -1.0), ambient=0.3, diffuse=0.7,
                    background=(0.2, 0.3, 0.4), geom_rgb=np.array([[0.6, 0.6, 0.6], [0.9, 0.3, 0.1]], np.float32))
    drawn = _check(m, scene, q.astype(np.float32), v.astype(np.float32), 12)
    assert drawn > 12 * 1500


def test_hidden_geoms_and_argument_errors():
    from paper_2502_08844_b300 import _capi
    m = W.cartpole_pixels()
    sc = W.cartpole_scene(32, 24)
    sc.geom_rgb = sc.geom_rgb.copy(); sc.geom_rgb[1, 0] = -1.0          # hide the pole
    run = GpuRun(m, 4)
    q, v = W.initial_state(m, 0, 4)
    run.set_state(q, v)
    _, hits = _render_gpu(run, sc, "f32")
    assert not np.any((hits & 0xFFFF) == 2)
    mixed = core.Batch([(core.CompiledModel(W.cartpole()), 2), (core.CompiledModel(W.quadruped()), 2)])
    st = core.State(mixed, "cuda")
    px = torch.zeros((4, 24, 32, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(_capi.PgError) as ei:
        core.render(mixed, st, sc, px)
    assert ei.value.code == _capi.PG_EUNSUPPORTED
    bad = W.cartpole_scene(0, 24)
    with pytest.raises(_capi.PgError) as ei:
        core.render(run.batch, run.state, bad, torch.zeros((4, 24, 0, 3), dtype=torch.uint8, device="cuda"))
    assert ei.value.code == _capi.PG_EINVAL


def test_visual_randomisation_matches_oracle():
    """Per-environment camera positions (look-at kept), light directions and colour tints: each
    image equals the oracle's image of that environment's scene, times its tint."""
    m = W.cartpole_pixels()
    n = 16
    sc = W.cartpole_scene(48, 40)
    q, v = W.initial_state(m, 0, n)
    q = q.copy(); q[:, 1] *= 8.0
    rng = np.random.default_rng(11)
    off = rng.uniform(-0.4, 0.4, (n, 3)).astype(np.float32)
    ldir = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.6, 0.6, n), -np.ones(n)], 1).astype(np.float32)
    tint = rng.uniform(0.6, 1.2, (n, 3)).astype(np.float32)
    run = GpuRun(m, n)
    run.set_state(q, v)
    ld = run.state.ld
    dev = lambda a: torch.from_numpy(core.to_soa(a, ld, 3)).to("cuda")
    px = torch.zeros((n, sc.height, sc.width, 3), dtype=torch.float32, device="cuda")
    hits = torch.zeros((n, sc.height, sc.width), dtype=torch.int32, device="cuda")
    core.render(run.batch, run.state, sc, px, hits, cam_offset=dev(off), light_dir=dev(ldir), tint=dev(tint))
    torch.cuda.synchronize()
    px, hits = px.cpu().numpy(), hits.cpu().numpy()
    om = O.OracleModel(m)
    differ = 0
    for e in range(n):
        oc, ocode = RD.render(om, RD.randomized_scene(sc, off[e], ldir[e]), q[e].astype(np.float64))
        oc = oc * tint[e].astype(np.float64)
        bad = hits[e] != ocode
        edge = _edge(ocode)
        assert not np.any(bad & ~edge), e
        differ += bad.sum()
        same = ~bad & ~edge
        # the camera basis is rebuilt per environment in float32 here (once per launch on the host
        # in float64 otherwise): ray directions carry a few ulps more, so 2e-4
        assert np.abs(px[e][same] - oc[same]).max() <= 2e-4, e
    assert differ <= 0.01 * n * sc.width * sc.height
    # the randomisation shows: two environments' backgrounds differ by their tints
    assert not np.allclose(px[0][hits[0] == 0].mean(0), px[1][hits[1] == 0].mean(0))
