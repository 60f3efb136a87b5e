"""Parity of the CUDA adjoint (pg_step_vjp behind torch.autograd) with the oracle's FP64
reverse-mode rollout gradient, itself pinned against FP64 central differences.

Both sides use the converged contact solver: its implicit derivative is what the adjoint
computes.  Gradients are compared norm-wise per quantity and environment at 1e-3 relative
(R19 form: max|g - g_ref| <= 1e-3 max|g_ref| + 1e-6)."""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_08844_b300 import adjoint, core
from paper_2502_08844_b300 import _capi
from paper_2502_08844_b300 import workloads as W

from tests import models_for_tests as MT

pytestmark = pytest.mark.gpu

GRAD_RTOL, GRAD_ATOL = 1e-3, 1e-6


def gpu_rollout_grad(m: W.Model, q0, v0, U, weights, segment=8, specialize=False):
    """GPU loss and per-env gradients of sum_t sum_i wq_i (q_t,i - qs_i)^2 + wv_i (v_t,i - vs_i)^2."""
    n, T = q0.shape[0], U.shape[0]
    cm = core.CompiledModel(m)
    batch = core.Batch([(cm, n)])
    if specialize:   # True: the branch-parallel step and tape where the model qualifies; "thread": not
        batch.specialize(branch=specialize != "thread")
        if specialize is True and cm.branch_plan()["branch"]:
            assert batch.kernel()["kernel"] == "branch-parallel"
    ld = max(4, (n + 3) // 4 * 4)
    dev = torch.device("cuda")
    qpos0 = torch.from_numpy(core.to_soa(q0.astype(np.float32), ld, batch.nq_max)).to(dev).requires_grad_()
    qvel0 = torch.from_numpy(core.to_soa(v0.astype(np.float32), ld, batch.nv_max)).to(dev).requires_grad_()
    ctrl_np = np.zeros((T, max(batch.nu_max, 1), ld), np.float32)
    ctrl_np[:, :m.nu, :n] = U.transpose(0, 2, 1)
    ctrl = torch.from_numpy(ctrl_np).to(dev).requires_grad_()
    params = adjoint.param_values(batch, ld, dev).requires_grad_()
    Q, V = adjoint.rollout(batch, qpos0, qvel0, ctrl, params, n_substeps=m.n_substeps, segment=segment)
    wq, qs, wv, vs = [torch.tensor(x, dtype=torch.float32, device=dev)[:, None] for x in weights]
    loss_env = ((wq * (Q[:, :m.nq, :n] - qs) ** 2).sum(dim=(0, 1)) + (wv * (V[:, :m.nv, :n] - vs) ** 2).sum(dim=(0, 1)))
    loss_env.sum().backward()
    torch.cuda.synchronize()
    nb, nv, nu = m.nbody, m.nv, m.nu
    gp = params.grad.cpu().numpy()[:, :n].T
    return {"loss": loss_env.detach().cpu().numpy().astype(np.float64),
            "traj_q": Q.detach().cpu().numpy()[:, :m.nq, :n].transpose(2, 0, 1).astype(np.float64),
            "traj_v": V.detach().cpu().numpy()[:, :m.nv, :n].transpose(2, 0, 1).astype(np.float64),
            "q0": qpos0.grad.cpu().numpy()[:m.nq, :n].T, "v0": qvel0.grad.cpu().numpy()[:nv, :n].T,
            "u": ctrl.grad.cpu().numpy()[:, :nu, :n].transpose(2, 0, 1), "mass": gp[:, :nb],
            "damping": gp[:, nb:nb + nv], "kp": gp[:, nb + nv:nb + nv + nu]}


def check_against_oracle(m, q0, v0, U, weights, keys=("q0", "v0", "u", "mass", "damping", "kp"), segment=8,
                         specialize=False):
    g = gpu_rollout_grad(m, q0, v0, U, weights, segment, specialize=specialize)
    om = O.OracleModel(m)
    worst = {}
    for e in range(q0.shape[0]):
        o = O.rollout_grad(om, q0[e].astype(np.float64), v0[e].astype(np.float64), U[:, e].astype(np.float64),
                           m.n_substeps, weights)
        assert abs(g["loss"][e] - o["loss"]) <= 1e-4 * abs(o["loss"]) + 1e-6, (e, g["loss"][e], o["loss"])
        for k in keys:
            ref = np.asarray(o[k], np.float64)
            if k == "mass":
                ref = ref[1:]
                x = g[k][e][1:]
            else:
                x = g[k][e]
            if ref.size == 0:
                continue
            scale = np.abs(ref).max()
            err = max(np.abs(x - ref).max() - GRAD_ATOL, 0.0) / max(scale, 1e-30)
            worst[k] = max(worst.get(k, 0.0), err)
            assert err <= GRAD_RTOL, "env %d %s: scaled error %.3e\ngpu %s\nref %s" % (e, k, err, x, ref)
    return worst


def _converged(m: W.Model) -> W.Model:
    return dataclasses.replace(m, iterations=100)


@pytest.mark.parametrize("specialize", [pytest.param(False, id="generic"), pytest.param("thread", id="specialised"),
                                        pytest.param(True, id="branch")])
def test_quadruped_rollout_gradient_matches_oracle(specialize):
    """End to end over one checkpoint segment (8 control steps = 40 substeps with contacts), with
    the library's compiled kernels, the model-specialised thread-per-environment ones, and the
    branch-parallel step and tape replay the benchmark times (the reverse sweep is the
    specialised one in both specialised cases)."""
    m = _converged(W.quadruped())
    n, T = 8, 8
    q0, v0 = W.initial_state(m, 4, n)
    U = W.actions(m, 4, n, 0, T)
    w = O.tracking_loss_weights(O.OracleModel(m))
    check_against_oracle(m, q0, v0, U, w, specialize=specialize)


def test_torque_limited_rollout_gradient_matches_oracle():
    """The quadruped with 4 Nm torque limits (its PD forces saturate): a clipped force is constant,
    so nothing flows back through it (kp and control gradients of a saturated actuator vanish);
    end to end over one segment against the oracle's reverse mode."""
    m = _converged(W.quadruped())
    m.act_forcelimited = np.ones(m.nu, np.int32)
    m.act_forcerange = np.tile(np.array([[-4.0, 4.0]], np.float32), (m.nu, 1))
    n, T = 8, 8
    q0, v0 = W.initial_state(m, 4, n)
    U = W.actions(m, 4, n, 0, T)
    w = O.tracking_loss_weights(O.OracleModel(m))
    check_against_oracle(m, q0, v0, U, w)


@pytest.mark.parametrize("specialize", [pytest.param(False, id="generic"), pytest.param(True, id="branch")])
def test_rough_terrain_rollout_gradient_matches_oracle(specialize):
    """The quadruped on gradient-noise terrain: its feet meet triangle faces, edges and vertices,
    where the contact normal turns with the state; end to end over one segment against the
    oracle's reverse mode, with the generic kernels and with the branch-parallel step and tape."""
    m = _converged(W.quadruped_rough())
    n, T = 8, 8
    q0, v0 = W.initial_state(m, 4, n)
    U = W.actions(m, 4, n, 0, T)
    w = O.tracking_loss_weights(O.OracleModel(m))
    check_against_oracle(m, q0, v0, U, w, specialize=specialize)


def _ball_on_terrain(elev):
    b = W.ModelBuilder("ball_terrain")
    g0 = b.geom(0, W.HFIELD, (0.2, 0.2, 0.1))
    ball = b.body(0, (0, 0, 0.2))
    b.joint(ball, W.FREE)
    g1 = b.geom(ball, W.SPHERE, (0.05,), mass=1.0)
    b.pair(g0, g1, friction=0.8, condim=3)
    return b.build(timestep=0.002, iterations=100, n_substeps=4, hfield=elev)


@pytest.mark.parametrize("feature", ["edge", "vertex"])
def test_terrain_edge_and_vertex_contact_gradients(feature):
    """A ball resting on a terrain ridge (its contact on a triangle edge) or on a peak (on a
    vertex): the normal follows the ball's centre, dn/dy = (I - n n^T)(I - u u^T) / |y - q| on the
    edge and (I - n n^T) / |y - q| at the vertex; against the oracle's reverse mode."""
    elev = np.zeros((5, 5), np.float32)
    if feature == "edge":
        elev[2, :] = 1.0            # a ridge along y = 0, 0.1 m high, 45-degree flanks
    else:
        elev[2, 2] = 1.0            # a peak at the origin
    m = _ball_on_terrain(elev)
    n, T = 4, 8
    q0 = np.zeros((n, 7))
    q0[:, 0] = [-0.02, 0.0, 0.01, 0.015] if feature == "edge" else [0.003, -0.002, 0.0, 0.004]
    q0[:, 1] = [0.0, 0.002, -0.004, 0.006] if feature == "edge" else [-0.002, 0.003, 0.001, 0.0]
    q0[:, 2] = 0.1495
    q0[:, 3] = 1.0
    v0 = np.zeros((n, 6))
    v0[:, 0] = [0.2, -0.1, 0.0, 0.3] if feature == "edge" else [0.0, 0.05, -0.05, 0.02]
    U = np.zeros((T, n, 0))
    w = O.tracking_loss_weights(O.OracleModel(m))
    check_against_oracle(m, q0, v0, U, w, keys=("q0", "v0", "mass"))


def test_cylinder_rollout_gradients_match_oracle():
    """Cylinders on a plane: one falling tilted and spinning (its deepest rim point slides round
    the rim as it turns), one rolling on its side and one landing upright on its tripod (rim points
    fixed to the body), against the oracle's reverse mode."""
    from tests.test_gpu_cylinder import _cylinder_scene, _initial_states
    m = dataclasses.replace(_cylinder_scene(), iterations=100)
    q0, v0 = _initial_states()
    T = 8
    U = np.zeros((T, 3, 0))
    w = O.tracking_loss_weights(O.OracleModel(m))
    check_against_oracle(m, q0, v0, U, w, keys=("q0", "v0", "mass"))


def test_upright_cylinder_landing_gradient_matches_central_differences():
    """A cylinder landing upright on its tripod, starting with zero angular velocity: the gradient
    with respect to the initial velocity against FP64 central differences of the oracle's loss
    (step 1e-6).  Its tilt derivative comes from the orientation update's derivative at w = 0."""
    from tests.test_gpu_cylinder import _cylinder_scene, _initial_states
    m = dataclasses.replace(_cylinder_scene(), iterations=100)
    q0, v0 = _initial_states()
    q0, v0 = q0[2:], v0[2:]
    T = 8
    U = np.zeros((T, 1, 0))
    om = O.OracleModel(m)
    w = O.tracking_loss_weights(om)
    g = gpu_rollout_grad(m, q0, v0, U, w)
    fd = np.zeros(6)
    for k in range(6):
        vp, vm = v0[0].copy(), v0[0].copy()
        vp[k] += 1e-6
        vm[k] -= 1e-6
        fd[k] = (O.rollout_loss(om, q0[0], vp, U[:, 0], m.n_substeps, w) -
                 O.rollout_loss(om, q0[0], vm, U[:, 0], m.n_substeps, w)) / 2e-6
    err = max(np.abs(g["v0"][0] - fd).max() - GRAD_ATOL, 0.0) / np.abs(fd).max()
    assert err <= GRAD_RTOL, (g["v0"][0], fd)
    assert abs(fd[4]) > 0.1          # the tilt the tripod's asymmetry sets up


def test_friction_loss_rollout_gradient_matches_oracle():
    """The quadruped with joint friction loss on its hinges: rows inside their band act as soft
    rows, rows at their bound pass nothing back; end to end over one segment against the oracle's
    reverse mode."""
    m = _converged(W.quadruped())
    m.dof_frictionloss = np.zeros(m.nv, np.float32)
    m.dof_frictionloss[6:] = 0.8
    n, T = 8, 8
    q0, v0 = W.initial_state(m, 4, n)
    U = W.actions(m, 4, n, 0, T)
    w = O.tracking_loss_weights(O.OracleModel(m))
    check_against_oracle(m, q0, v0, U, w)


def _contact_states(m, n_states=8, T=60):
    """FP32 quadruped states along an oracle rollout (standing, stepping, sliding contacts)."""
    om = O.OracleModel(m)
    q0, v0 = W.initial_state(m, 4, 4)
    U = W.actions(m, 4, 4, 0, T)
    _, _, _, _, tq, tv = om.rollout(q0, v0, U, m.n_substeps, solver_cap=-1, trajectory=True)
    ts = np.linspace(0, T - 2, n_states).astype(int)
    q = np.stack([tq[t, i % 4] for i, t in enumerate(ts)]).astype(np.float32).astype(np.float64)
    v = np.stack([tv[t, i % 4] for i, t in enumerate(ts)]).astype(np.float32).astype(np.float64)
    u = np.stack([U[t + 1, i % 4] for i, t in enumerate(ts)])
    return q, v, u


def test_single_control_step_vjp_at_contact_states():
    """One control step (5 substeps) backward from states with different contact sets: the FP32
    adjoint against the FP64 reverse mode at 1e-4 (observed ~1e-6: only rounding separates them)."""
    m = _converged(W.quadruped())
    q0, v0, u = _contact_states(m)
    w = O.tracking_loss_weights(O.OracleModel(m))
    g = gpu_rollout_grad(m, q0, v0, u[None].astype(np.float32), w)
    om = O.OracleModel(m)
    for e in range(q0.shape[0]):
        o = O.rollout_grad(om, q0[e], v0[e], u[e][None], m.n_substeps, w)
        for k in ("q0", "v0", "u", "mass", "damping", "kp"):
            ref = np.asarray(o[k], np.float64).ravel()
            x = g[k][e].ravel()
            if k == "mass":
                ref, x = ref[1:], x[1:]
            err = max(np.abs(x - ref).max() - GRAD_ATOL, 0.0) / np.abs(ref).max()
            assert err <= 1e-4, (e, k, err)


@pytest.mark.parametrize("T,specialize", [(16, False), (64, False), (64, "thread"), (64, True)])
def test_quadruped_rollout_reanchored_on_gpu_trajectory(T, specialize):
    """Two and eight checkpoint segments (16 and 64 control steps: the adjoint workload's horizon).
    The oracle's per-step reverse sweep is chained along the GPU's own FP32 trajectory, so the
    comparison measures the adjoint, not the divergence of FP32 and FP64 forward rollouts through
    contact events."""
    m = _converged(W.quadruped())
    n = 8
    q0, v0 = W.initial_state(m, 4, n)
    q0 = q0.astype(np.float64); v0 = v0.astype(np.float64)
    U = W.actions(m, 4, n, 0, T)
    w = O.tracking_loss_weights(O.OracleModel(m))
    wq, qs, wv, vs = w
    g = gpu_rollout_grad(m, q0, v0, U, w, specialize=specialize)
    Q, V = g["traj_q"], g["traj_v"]            # [n, T, nq], the GPU states after each step
    om = O.OracleModel(m)
    for e in range(n):
        Qe = np.concatenate([q0[e][None], Q[e]]); Ve = np.concatenate([v0[e][None], V[e]])
        bq = np.zeros(m.nq); bv = np.zeros(m.nv)
        gu = np.zeros((T, m.nu)); gm = np.zeros(m.nbody); gd = np.zeros(m.nv); gk = np.zeros(m.nu)
        for t in range(T - 1, -1, -1):
            bq = bq + 2 * wq * (Qe[t + 1] - qs); bv = bv + 2 * wv * (Ve[t + 1] - vs)
            o = O.step_vjp(om, Qe[t], Ve[t], U[t, e], m.n_substeps, bq, bv)
            bq, bv, gu[t] = o["q"], o["v"], o["u"]
            gm += o["mass"]; gd += o["damping"]; gk += o["kp"]
        for k, ref in (("q0", bq), ("v0", bv), ("u", gu), ("mass", gm[1:]), ("damping", gd), ("kp", gk)):
            x = g[k][e][1:] if k == "mass" else g[k][e]
            err = max(np.abs(x - ref).max() - GRAD_ATOL, 0.0) / np.abs(ref).max()
            assert err <= GRAD_RTOL, (e, k, err)


def test_cartpole_rollout_gradient_matches_oracle():
    m = W.cartpole()
    n, T = 8, 16
    q0, v0 = W.initial_state(m, 0, n)
    U = W.actions(m, 0, n, 0, T)
    om = O.OracleModel(m)
    w = (np.ones(m.nq), np.zeros(m.nq), np.ones(m.nv), np.zeros(m.nv))
    check_against_oracle(m, q0, v0, U, w, keys=("q0", "v0", "u", "mass", "damping"))


def box_capsule_states(n, seed=7):
    """Tilted box and capsule whose lowest corner / end is 1 mm inside the floor, small random
    velocities: box-corner and capsule-end contacts active through the rollout."""
    rng = np.random.default_rng(seed)
    q0 = np.zeros((n, 14)); v0 = np.zeros((n, 12))
    corners = np.array([[sx, sy, sz] for sx in (-0.05, 0.05) for sy in (-0.04, 0.04) for sz in (-0.03, 0.03)])
    ends = np.array([[0, 0, -0.08], [0, 0, 0.08]])
    for e in range(n):
        for b, (x, pts, rad) in enumerate([(0.0, corners, 0.0), (0.5, ends, 0.02)]):
            ax = rng.normal(size=3); ax /= np.linalg.norm(ax)
            ang = rng.uniform(0.1, 0.5)
            qw, qv = np.cos(ang / 2), np.sin(ang / 2) * ax
            R = (2 * qw * qw - 1) * np.eye(3) + 2 * np.outer(qv, qv) + 2 * qw * np.array(
                [[0, -qv[2], qv[1]], [qv[2], 0, -qv[0]], [-qv[1], qv[0], 0]])
            z = -(pts @ R.T)[:, 2].min() + rad - 0.001
            q0[e, 7 * b:7 * b + 7] = [x, 0.0, z, qw, *qv]
            v0[e, 6 * b:6 * b + 6] = rng.normal(scale=0.05, size=6)
    return q0.astype(np.float32).astype(np.float64), v0.astype(np.float32).astype(np.float64)


def test_box_and_capsule_contact_features_gradient():
    m = MT.box_and_capsule_on_plane()
    n, T = 6, 12
    q0, v0 = box_capsule_states(n)
    U = np.zeros((T, n, 0))
    w = (np.r_[[0, 0, 1.0] + [0] * 4 + [0, 0, 1.0] + [0] * 4], np.zeros(m.nq), np.ones(m.nv), np.zeros(m.nv))
    check_against_oracle(m, q0, v0, U, w, keys=("q0", "v0"))
    # scaling a lone body's mass (and with it its inertia) scales M and D = d / ((1 - d) Ahat),
    # Ahat ~ 1/m, alike: the accelerations, hence the loss, do not depend on it.  The FP32
    # gradient is zero up to the rounding of its terms.
    g = gpu_rollout_grad(m, q0, v0, U, w)
    assert np.abs(g["mass"][:, 1:]).max() <= 1e-6 * np.abs(g["q0"]).max()


def test_joint_limit_rows_gradient():
    m = MT.limited_arm()
    n, T = 6, 20
    rng = np.random.default_rng(3)
    q0 = rng.uniform(-0.3, 0.25, size=(n, m.nq)).astype(np.float32).astype(np.float64)
    v0 = rng.normal(scale=0.5, size=(n, m.nv)).astype(np.float32).astype(np.float64)
    U = np.stack([np.array([[0.8, -0.9]] * n) + 0.05 * rng.normal(size=(n, 2)) for _ in range(T)]).astype(np.float32)
    w = (np.ones(m.nq), np.zeros(m.nq), np.ones(m.nv), np.zeros(m.nv))
    check_against_oracle(m, q0, v0, U, w)


def test_segment_length_does_not_change_the_gradient():
    m = _converged(W.quadruped())
    n, T = 4, 12
    q0, v0 = W.initial_state(m, 4, n)
    U = W.actions(m, 4, n, 0, T)
    w = O.tracking_loss_weights(O.OracleModel(m))
    a = gpu_rollout_grad(m, q0, v0, U, w, segment=8)
    b = gpu_rollout_grad(m, q0, v0, U, w, segment=5)
    for k in ("q0", "v0", "u", "mass", "damping", "kp"):
        assert np.array_equal(a[k], b[k]), k


def test_vjp_rejects_models_outside_scope():
    hand = core.CompiledModel(W.hand())
    assert hand.sizes.adjoint_workspace_bytes == 0
    batch = core.Batch([(hand, 4)])
    st = core.State(batch)
    ld = st.ld
    dev = st.qpos.device
    ctrl = torch.zeros((1, batch.nu_max, ld), device=dev)
    with pytest.raises(_capi.PgError) as ei:
        core.step_vjp(batch, st, ctrl, 0, None, None, torch.zeros_like(st.qpos), torch.zeros_like(st.qvel),
                      torch.zeros_like(ctrl), torch.zeros((batch.nparam_max, ld), device=dev))
    assert ei.value.code == _capi.PG_EUNSUPPORTED
