"""GPU parity of cylinder-plane contacts against the FP64 oracle, through the C ABI: every phase
of a substep on contact states of a cylinder that falls tilted, rolls on its side and lands on
its cap; 40-step rollouts at the rollout tolerance; and the model-specialised kernel against the
generic one."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_08844_b300 import core, workloads as W
from tests.gpu_helpers import GpuRun, canon_qpos
from tests.test_gpu_hfield import _rounding_sensitivity
from tests.test_gpu_parity import ONE_STEP_RTOL, ROLLOUT_RTOL, assert_close_scaled

pytestmark = pytest.mark.gpu

R, HL = 0.06, 0.1


def _cylinder_scene():
    b = W.ModelBuilder("cylinder_plane")
    g0 = b.geom(0, W.PLANE, (0, 0, 0))
    body = b.body(0, (0, 0, 0.2))
    b.joint(body, W.FREE)
    g1 = b.geom(body, W.CYLINDER, (R, HL), mass=1.0)
    b.pair(g0, g1, friction=0.8, condim=3)
    m = b.build(timestep=0.002, iterations=6, n_substeps=4)
    m.qpos_init = W._f32([0, 0, 0.2, 1, 0, 0, 0])
    return m


def _initial_states():
    """Three starts: tilted 0.5 rad and spinning a little, lying on its side and rolling, and
    upright just above the plane (it lands on its tripod)."""
    c, s = math.cos(0.25), math.sin(0.25)
    h = math.sqrt(0.5)
    q0 = np.array([[0.0, 0.0, HL * math.cos(0.5) + R * math.sin(0.5) + 0.01, c, s, 0.0, 0.0],
                   [0.3, 0.1, R + 0.002, h, h, 0.0, 0.0],
                   [-0.2, 0.0, HL + 0.004, 1.0, 0.0, 0.0, 0.0]])
    v0 = np.zeros((3, 6))
    v0[0, 3:6] = [0.0, 0.4, 1.5]
    v0[1, 0], v0[1, 4] = 0.5, 0.5 / R
    return q0, v0


def test_cylinder_phase_parity():
    m = _cylinder_scene()
    om = O.OracleModel(m)
    q0, v0 = _initial_states()
    U = np.zeros((80, 3, 0))
    _, _, _, _, tq, tv = om.rollout(q0, v0, U, 4, trajectory=True)
    ncon = {e: [] for e in range(3)}
    for t in (20, 45, 79):
        for e in range(3):
            q = tq[t, e].astype(np.float32).astype(np.float64)
            v = tv[t, e].astype(np.float32).astype(np.float64)
            run = GpuRun(m, 3)
            run.set_state(np.repeat(q[None], 3, 0), np.repeat(v[None], 3, 0))
            g = run.debug(np.zeros((3, 0)), e)
            o = om.forward(q, v, np.zeros(6), np.zeros(0))
            for k in ("xpos", "xmat", "M", "bias", "a0"):
                assert_close_scaled(k, g[k], o[k], ONE_STEP_RTOL)
            assert np.array_equal(g["contacts"][:, 0], o["contacts"][:, 0])
            for a, b, name in [(1, 2, "dist"), (2, 5, "pos"), (5, 14, "frame")]:
                assert_close_scaled("contact " + name, g["contacts"][:, a:b], o["contacts"][:, a:b], ONE_STEP_RTOL)
            assert g["nrow"] == o["nrow"]
            if g["nrow"]:
                assert_close_scaled("J", g["rows"][:, :6], o["rows"][:, :6], ONE_STEP_RTOL)
            # resting on two or three rim points makes the solve as ill-conditioned as a capsule
            # on both end spheres: qacc is held to 4x the oracle's own sensitivity to one float32
            # rounding of the state (at least the one-step tolerance)
            tol = max(ONE_STEP_RTOL, 4.0 * _rounding_sensitivity(om, q, v))
            assert_close_scaled("qacc", g["qacc"], o["qacc"], tol)
            vscale = max(np.abs(o["qvel_next"]).max(), m.timestep * np.abs(o["qacc"]).max())
            assert_close_scaled("qvel_next", g["qvel_next"], o["qvel_next"], ONE_STEP_RTOL, vscale)
            assert_close_scaled("qpos_next", canon_qpos(m, g["qpos_next"]), canon_qpos(m, o["qpos_next"]),
                                ONE_STEP_RTOL)
            ncon[e].append(int(o["contacts"][:, 0].sum()))
    assert max(ncon[1]) == 2          # on its side: both rims
    assert ncon[2][-1] == 3           # upright: the tripod
    assert max(ncon[0]) >= 1


def test_cylinder_rollout_parity():
    m = _cylinder_scene()
    om = O.OracleModel(m)
    q0, v0 = _initial_states()
    q0, v0 = q0.astype(np.float32), v0.astype(np.float32)
    run = GpuRun(m, 3)
    run.set_state(q0, v0)
    T = 40
    tqg, tvg = run.rollout(np.zeros((T, 3, 0), np.float32), 4, keep=True)
    qo, vo, _, _ = om.rollout(q0, v0, np.zeros((T, 3, 0)), 4)
    for e in range(3):
        assert_close_scaled("qpos env %d" % e, canon_qpos(m, tqg[-1, e]), canon_qpos(m, qo[e]), ROLLOUT_RTOL)
        assert_close_scaled("qvel env %d" % e, tvg[-1, e], vo[e], ROLLOUT_RTOL)


def test_specialised_cylinder_matches_generic():
    import torch
    m = _cylinder_scene()
    q0, v0 = _initial_states()
    n = 96
    q0 = np.repeat(q0, n // 3, 0)
    v0 = np.repeat(v0, n // 3, 0)
    q0[:, 0] += np.linspace(-0.1, 0.1, n)
    outs = []
    for spec in (False, True):
        cm = core.CompiledModel(m)
        batch = core.Batch([(cm, n)])
        if spec:
            batch.specialize()
        st = core.State(batch, "cuda:0")
        st.qpos.copy_(torch.from_numpy(core.to_soa(q0, st.ld, batch.nq_max)))
        st.qvel.copy_(torch.from_numpy(core.to_soa(v0, st.ld, batch.nv_max)))
        ctrl = torch.zeros((1, st.ld), device="cuda:0")
        for _ in range(10):
            core.step(batch, st, ctrl, 4)
        torch.cuda.synchronize()
        outs.append((st.qpos.cpu().numpy(), st.qvel.cpu().numpy()))
    for a, b in zip(outs[0], outs[1]):
        assert np.allclose(a, b, rtol=1e-4, atol=1e-5)
