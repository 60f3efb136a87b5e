"""GPU parity of heightfield contacts (rough terrain) against the FP64 oracle, through the C ABI:
every phase of a substep on contact states of the quadruped on gradient-noise terrain, one
control step and 50-step rollouts at the step tolerances, a capsule on the terrain, and the
model-specialised kernel against the generic one.  The contact tolerances are the plane's:
the heightfield adds a triangle search whose result is continuous in the state."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_08844_b300 import core, workloads as W
from tests.gpu_helpers import GpuRun, canon_qpos
from tests.test_gpu_parity import (ONE_STEP_RTOL, ROLLOUT_RTOL, _phase_compare, _rollout_states, _trajectory_parity,
                                   assert_close_scaled)

pytestmark = pytest.mark.gpu


def test_phase_parity_rough_terrain():
    m = W.quadruped_rough()
    om, states = _rollout_states(m, 1, (0, 12, 30, 60))
    nrows = []
    for q, v, u in states:
        g, o = _phase_compare(m, om, q, v, u, env=1, n=4)
        nrows.append(g["nrow"])
        n = o["contacts"][:, 5:8]
        assert np.all(np.abs(n[:, 2]) > 0.9)           # terrain normals, not all vertical
    assert max(nrows) >= 8


@pytest.mark.parametrize("n,T,rtol", [(37, 1, ONE_STEP_RTOL), (33, 50, ROLLOUT_RTOL)])
def test_rough_terrain_trajectories(n, T, rtol):
    m, tqg, tvg, tqo, tvo, stg, sto = _trajectory_parity("quadruped_rough", 1, n, T)
    for e in range(n):
        assert_close_scaled("qpos env %d" % e, canon_qpos(m, tqg[-1, e]), canon_qpos(m, tqo[-1, e]), rtol)
        assert_close_scaled("qvel env %d" % e, tvg[-1, e], tvo[-1, e], rtol)


def _capsule_on_terrain():
    b = W.ModelBuilder("capsule_terrain")
    hf = W.perlin_terrain(21, 25, 4, seed=11)
    g0 = b.geom(0, W.HFIELD, (1.2, 1.0, 0.08))
    body = b.body(0, (0.1, -0.05, 0.2), quat=(0.9, 0.1, 0.3, 0.0))
    b.joint(body, W.FREE)
    g1 = b.geom(body, W.CAPSULE, (0.03, 0.15), mass=1.0)
    b.pair(g0, g1, friction=0.8, condim=3)
    m = b.build(timestep=0.002, iterations=6, n_substeps=4, hfield=hf)
    m.qpos_init = W._f32([0.1, -0.05, 0.2, 0.9, 0.1, 0.3, 0.0])
    return m


def _rounding_sensitivity(om, q, v, trials=12, seed=0):
    """Largest relative change of the oracle's qacc when q and v are perturbed by one float32
    rounding (relative 2^-24): what FP32 input rounding alone does to the solve."""
    rng = np.random.default_rng(seed)
    o = om.forward(q, v, np.zeros(om.nv), np.zeros(0))["qacc"]
    worst = 0.0
    for _ in range(trials):
        e = 2.0 ** -24
        op = om.forward(q * (1 + rng.uniform(-e, e, q.shape)), v * (1 + rng.uniform(-e, e, v.shape)),
                        np.zeros(om.nv), np.zeros(0))["qacc"]
        worst = max(worst, np.abs(op - o).max() / np.abs(o).max())
    return worst


def test_capsule_on_terrain_phases_and_rollout():
    """A capsule resting on both end spheres makes the contact solve ill-conditioned: one float32
    rounding of the input state moves the oracle's own qacc by 1e-5 - 6e-5 of its scale.  qacc
    is therefore held to 4x that measured sensitivity (at least the one-step 1e-5); the contact
    geometry, the Jacobian rows and the next qpos / qvel keep the one-step tolerance."""
    m = _capsule_on_terrain()
    om = O.OracleModel(m)
    q0 = np.tile(m.qpos_init.astype(np.float64), (3, 1))
    q0[:, 0] += [0.0, 0.3, -0.4]
    v0 = np.zeros((3, 6)); v0[:, 0] = [0.5, -0.2, 0.1]
    U = np.zeros((80, 3, 0))
    _, _, _, _, tq, tv = om.rollout(q0, v0, U, 4, trajectory=True)
    nrows = []
    for t in (30, 50, 79):
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
            tol = max(ONE_STEP_RTOL, 4.0 * _rounding_sensitivity(om, q, v))
            assert_close_scaled("qacc", g["qacc"], o["qacc"], tol)
            vscale = max(np.abs(o["qvel_next"]).max(), m.timestep * np.abs(o["qacc"]).max())
            assert_close_scaled("qvel_next", g["qvel_next"], o["qvel_next"], ONE_STEP_RTOL, vscale)
            assert_close_scaled("qpos_next", canon_qpos(m, g["qpos_next"]), canon_qpos(m, o["qpos_next"]), ONE_STEP_RTOL)
            nrows.append(g["nrow"])
    assert max(nrows) >= 8                                # both end spheres down
    run = GpuRun(m, 3)
    run.set_state(q0.astype(np.float32), v0.astype(np.float32))
    tqg, tvg = run.rollout(np.zeros((40, 3, 0), np.float32), 4, keep=True)
    qo, vo, _, _ = om.rollout(q0.astype(np.float32), v0.astype(np.float32), U[:40], 4)
    for e in range(3):
        assert_close_scaled("qpos", canon_qpos(m, tqg[-1, e]), canon_qpos(m, qo[e]), ROLLOUT_RTOL)


def test_specialised_rough_terrain_matches_generic():
    """the specialised thread-per-environment kernel against the generic one (the same code, to
    rounding; the branch-parallel kernel on the terrain is checked against the oracle in
    test_gpu_branch.py)"""
    import torch
    m = W.quadruped_rough()
    outs = []
    for spec in (False, True):
        cm = core.CompiledModel(m)
        batch = core.Batch([(cm, 300)])
        if spec:
            batch.specialize(branch=False)
        st = core.State(batch, "cuda:0")
        q0, v0 = W.initial_state(m, 1, 300)
        st.qpos.copy_(torch.from_numpy(core.to_soa(q0, st.ld, batch.nq_max)))
        st.qvel.copy_(torch.from_numpy(core.to_soa(v0, st.ld, batch.nv_max)))
        U = W.actions(m, 1, 300, 0, 10)
        for t in range(10):
            core.step(batch, st, torch.from_numpy(core.to_soa(U[t], st.ld, batch.nu_max)).to("cuda:0"), 5)
        torch.cuda.synchronize()
        outs.append((st.qpos.cpu().numpy(), st.qvel.cpu().numpy()))
    for a, b in zip(outs[0], outs[1]):
        assert np.allclose(a, b, rtol=1e-4, atol=1e-5)
