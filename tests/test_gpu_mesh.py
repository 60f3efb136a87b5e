"""GPU parity of convex meshes and solid contacts against the FP64 oracle through the C ABI: the
seeded convex hulls dropped on a plane and on a heightfield (plane-mesh and heightfield-mesh
pairs, the hulls' mass properties in M), and the humanoid's box feet on rough terrain
(heightfield-box pairs): every substep phase at contact states, one control step and rollouts,
generic and specialised kernels."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_08844_b300 import workloads as W
from tests.gpu_helpers import GpuRun, canon_qpos
from tests.test_gpu_parity import ONE_STEP_RTOL, ROLLOUT_RTOL, ROW_DERIVED_RTOL, PHASE_FIELDS, assert_close_scaled

pytestmark = pytest.mark.gpu

# (model, input config, initial-state noise): the hulls start perturbed (positions, orientations and
# velocities U(+-0.02), clear of the ground) and fall; the humanoid from its reference pose under
# random PD targets
MODELS = {"hulls": (5, 0.02), "humanoid_rough": (3, 0.0)}


def _start(m, n):
    cfg, noise = MODELS[m.name]
    return W.initial_state(m, cfg, n, noise=noise)


def _controls(m, n, T):
    cfg, _ = MODELS[m.name]
    return W.actions(m, cfg, n, 0, T) if m.nu else np.zeros((T, n, 0), np.float32)


def _states(m, times, n_env=3):
    om = O.OracleModel(m)
    q0, v0 = _start(m, n_env)
    T = max(times) + 2
    U = _controls(m, n_env, T)
    _, _, _, _, tq, tv = om.rollout(q0, v0, U, m.n_substeps, trajectory=True, nthreads=4)
    out = []
    for t in times:
        for e in range(n_env):
            out.append((tq[t, e].astype(np.float32).astype(np.float64), tv[t, e].astype(np.float32).astype(np.float64),
                        U[t + 1, e].astype(np.float64)))
    return om, out


def _fields(o, nv):
    return {"a0": o["a0"], "qacc": o["qacc"], "aref": o["rows"][: o["nrow"], nv + 2]}


def _sensitivity(om, q, v, u, trials=8, seed=0):
    """for a0, qacc and the rows' aref: the largest change of the oracle's own result (relative to
    its largest entry) when q, v and u are moved by one float32 rounding (relative 2^-24), what
    FP32 input rounding alone does to it"""
    rng = np.random.default_rng(seed)
    o = _fields(om.forward(q, v, np.zeros(om.nv), u), om.nv)
    e = 2.0 ** -24
    worst = dict.fromkeys(o, 0.0)
    for _ in range(trials):
        p = lambda x: x * (1 + rng.uniform(-e, e, np.shape(x)))
        op = _fields(om.forward(p(q), p(v), np.zeros(om.nv), p(u)), om.nv)
        for k in o:
            if op[k].shape == o[k].shape and o[k].size:
                worst[k] = max(worst[k], np.abs(op[k] - o[k]).max() / max(np.abs(o[k]).max(), 1e-30))
    return worst


def _check_a0(m, g, o, trials=8, seed=0):
    """a0 = M^-1 (tau - c), an FP32 solve: within the larger of the one-step tolerance and 4x the
    solve's own sensitivity to FP32 rounding of its data -- the largest relative change of the
    FP64 solution when every entry of M (kept symmetric) and of the passive, actuator and bias
    forces moves by a relative U(+-2^-24) -- the size of error FP32 makes where the fallen
    humanoid's M (cond 7e3) meets PD and bias forces that largely cancel."""
    x, ref = np.asarray(g["a0"], np.float64), np.asarray(o["a0"], np.float64)
    M = np.asarray(o["M"], np.float64).reshape(m.nv, m.nv)
    parts = [np.asarray(o[k], np.float64) for k in ("passive", "actuator", "bias")]
    rng = np.random.default_rng(seed)
    e = 2.0 ** -24
    p = lambda x: x * (1 + rng.uniform(-e, e, x.shape))
    sens = 0.0
    for _ in range(trials):
        P = rng.uniform(-e, e, M.shape)
        Mp = M * (1 + (P + P.T) / 2)
        xp = np.linalg.solve(Mp, p(parts[0]) + p(parts[1]) - p(parts[2]))
        sens = max(sens, np.abs(xp - ref).max() / np.abs(ref).max())
    assert_close_scaled("a0", x, ref, max(ONE_STEP_RTOL, 4.0 * sens))


def _check_qacc(m, g, o, tol):
    """qacc, the minimiser of the soft-contact cost: within tol of the oracle's, or else a
    stationary point of the oracle's own cost to a backward error of 1e-5 -- the gradient
    M (a - a0) + sum over active rows of D (J a - aref) J in FP64 at the GPU's a (the active set
    taken there, the pyramid's one-sided rows), against the sum of its terms' magnitudes -- which is
    what the Newton step's FP32 linear solve guarantees; its forward error then depends on the
    conditioning of H = M + J_A^T D J_A (the fallen humanoid's)."""
    x, ref = np.asarray(g["qacc"], np.float64), np.asarray(o["qacc"], np.float64)
    if np.abs(x - ref).max() - 1e-6 <= tol * np.abs(ref).max():
        return
    assert m.cone == W.PYRAMIDAL and m.dof_frictionloss is None
    nv = m.nv
    M = np.asarray(o["M"], np.float64).reshape(nv, nv)
    t = x - np.asarray(o["a0"], np.float64)
    r, scale = M @ t, np.abs(M) @ np.abs(t)
    rows = np.asarray(o["rows"], np.float64)[: o["nrow"]]
    for J, aref, D in zip(rows[:, :nv], rows[:, nv + 2], rows[:, nv + 3]):
        res = J @ x - aref
        if res < 0:
            r += D * res * J
            scale += D * abs(res) * np.abs(J)
    assert np.abs(r).max() <= ONE_STEP_RTOL * scale.max(), ("qacc backward error", np.abs(r).max(), scale.max())


@pytest.mark.parametrize("mname", sorted(MODELS))
def test_phase_parity_solid_contacts(mname):
    """kinematics, M (the hulls' mass properties), bias and actuation, the contacts slot by slot
    (solid candidates in candidate order), rows, forces and the next state, at states along a
    rollout, at the one-step tolerance.  Where FP32 cannot resolve the one-step tolerance, the
    bound is what FP32 can: qacc and the rows' aref are held to the larger of their tolerance and
    4x the oracle's own sensitivity to one float32 rounding of the inputs (a light hull on stiff
    contacts amplifies input rounding); a0 and qacc as _check_a0 and _check_qacc say."""
    m = W.model(mname)
    # the hulls falling, landing and settling; the humanoid on its feet (its contact phase)
    om, states = _states(m, (0, 40, 80) if mname == "hulls" else (6, 20, 45))
    active = 0
    for q, v, u in states:
        n = 4
        run = GpuRun(m, n)
        run.set_state(np.repeat(q[None], n, 0), np.repeat(v[None], n, 0))
        g = run.debug(np.repeat(u[None], n, 0), 1)
        o = om.forward(q, v, np.zeros(m.nv), u)
        sens = _sensitivity(om, q, v, u)
        for k in PHASE_FIELDS:
            if k == "a0":
                _check_a0(m, g, o)
                continue
            if k == "qacc":
                _check_qacc(m, g, o, max(ONE_STEP_RTOL, 4.0 * sens["qacc"]))
                continue
            tol = max(ONE_STEP_RTOL, 4.0 * sens[k]) if k in sens else ONE_STEP_RTOL
            assert_close_scaled(k, g[k], o[k], tol)
        assert np.array_equal(g["contacts"][:, 0], o["contacts"][:, 0])
        for a, b, name in [(1, 2, "dist"), (2, 5, "pos"), (5, 14, "frame")]:
            assert_close_scaled("contact " + name, g["contacts"][:, a:b], o["contacts"][:, a:b], ONE_STEP_RTOL)
        assert g["nrow"] == o["nrow"]
        if g["nrow"]:
            assert_close_scaled("J", g["rows"][:, :m.nv], o["rows"][:, :m.nv], ONE_STEP_RTOL)
            for i, k in enumerate(["r", "v", "aref", "D", "Ahat", "imp"]):
                tol = ROW_DERIVED_RTOL.get(k, ONE_STEP_RTOL)
                if k == "aref":
                    tol = max(tol, 4.0 * sens["aref"])
                assert_close_scaled(k, g["rows"][:, m.nv + i], o["rows"][:, m.nv + i], tol)
        vscale = max(np.abs(o["qvel_next"]).max(), m.timestep * np.abs(o["qacc"]).max())
        assert_close_scaled("qvel_next", g["qvel_next"], o["qvel_next"], max(ONE_STEP_RTOL, 4.0 * sens["qacc"]), vscale)
        assert_close_scaled("qpos_next", canon_qpos(m, g["qpos_next"]), canon_qpos(m, o["qpos_next"]), ONE_STEP_RTOL)
        active = max(active, int((o["contacts"][:, 0] > 0).sum()))
    assert active >= 3                   # solid contacts were exercised


@pytest.mark.parametrize("specialize", [pytest.param(False, id="generic"), pytest.param(True, id="specialised")])
@pytest.mark.parametrize("mname,n,T,rtol", [("hulls", 33, 1, ONE_STEP_RTOL), ("hulls", 24, 20, ROLLOUT_RTOL),
                                            ("humanoid_rough", 33, 1, ONE_STEP_RTOL),
                                            ("humanoid_rough", 16, 30, ROLLOUT_RTOL)])
def test_solid_contact_trajectories(mname, n, T, rtol, specialize):
    m = W.model(mname)
    om = O.OracleModel(m)
    q0, v0 = _start(m, n)
    U = _controls(m, n, T)
    run = GpuRun(m, n, specialize=specialize)
    run.set_state(q0, v0)
    run.rollout(U, m.n_substeps)
    qg, vg, _ = run.get()
    qo, vo, _, _ = om.rollout(q0, v0, U, m.n_substeps, nthreads=8)
    for e in range(n):
        assert_close_scaled("qpos env %d" % e, canon_qpos(m, qg[e]), canon_qpos(m, qo[e]), rtol)
        assert_close_scaled("qvel env %d" % e, vg[e], vo[e], rtol)


@pytest.mark.parametrize("specialize", [pytest.param(False, id="generic"), pytest.param(True, id="specialised")])
def test_hulls_50_steps_reanchored(specialize):
    """The hulls over 50 control steps (they fall, land, tumble and settle), each step compared with
    the oracle's step from the GPU's own state: qpos at the one-step tolerance, qvel at the larger
    of it and 4x the oracle's own sensitivity of that step to one float32 rounding of its inputs.
    Free-running, tumbling contact dynamics separate FP32 and FP64 trajectories (20 steps hold 1e-3,
    test above); re-anchored, each step's arithmetic is checked."""
    m = W.hulls()
    om = O.OracleModel(m)
    n, T = 12, 50
    q0, v0 = _start(m, n)
    run = GpuRun(m, n, specialize=specialize)
    run.set_state(q0, v0)
    q, v, w = q0.astype(np.float64), v0.astype(np.float64), np.zeros((n, m.nv))
    U = np.zeros((1, n, 0))
    rng = np.random.default_rng(1)
    e = 2.0 ** -24
    for t in range(T):
        run.step(np.zeros((n, 0), np.float32), m.n_substeps)
        qg, vg, wg = run.get()
        qo, vo, _, _ = om.rollout(q, v, U, m.n_substeps, qacc_warm=w, nthreads=8)
        sens = np.zeros(n)
        for _ in range(3):
            p = lambda x: x * (1 + rng.uniform(-e, e, np.shape(x)))
            _, vp, _, _ = om.rollout(p(q), p(v), U, m.n_substeps, qacc_warm=w, nthreads=8)
            sens = np.maximum(sens, np.abs(vp - vo).max(axis=1) / np.maximum(np.abs(vo).max(axis=1), 1e-30))
        for k in range(n):
            assert_close_scaled("step %d qpos env %d" % (t, k), canon_qpos(m, qg[k]), canon_qpos(m, qo[k]), ONE_STEP_RTOL)
            assert_close_scaled("step %d qvel env %d" % (t, k), vg[k], vo[k], max(ONE_STEP_RTOL, 4.0 * sens[k]))
        q, v, w = qg, vg, wg


def test_solid_pairs_are_outside_the_adjoint():
    """mesh and heightfield-box pairs are outside the adjoint's scope; the humanoid's box feet on
    the terrain run the branch-parallel kernel, the free hulls (no branch) do not"""
    from paper_2502_08844_b300 import core
    for mname in MODELS:
        assert core.CompiledModel(W.model(mname)).sizes.adjoint_workspace_bytes == 0
    assert core.CompiledModel(W.humanoid_rough()).branch_plan()["branch"]
    assert not core.CompiledModel(W.hulls()).branch_plan()["branch"]
