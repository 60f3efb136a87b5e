"""pg_batch_specialize: the step kernel compiled at run time (NVRTC) with the model as constants
runs the same source as the generic kernel.  With the model known the compiler may fold known
zeros and forward stored constants, which can regroup an FMA, so trajectories agree to rounding
(1e-6 of their scale over a few steps; often bitwise).  Mixed batches keep the generic kernel."""
import numpy as np
import pytest
import torch

from paper_2502_08844_b300 import _capi, core
from paper_2502_08844_b300 import workloads as W
from tests.gpu_helpers import GpuRun

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mname,cfg,n,T", [("quadruped", 1, 300, 6), ("cartpole", 0, 77, 6), ("hand_elliptic", 2, 40, 3),
                                          ("humanoid", 3, 50, 3)])
def test_specialised_kernel_matches_generic(mname, cfg, n, T):
    m = W.model(mname)
    q0, v0 = W.initial_state(m, cfg, n)
    U = W.actions(m, cfg, n, 0, T)
    out = []
    for spec in (False, True):
        run = GpuRun(m, n)
        if spec:
            run.batch.specialize(branch=False)
        run.set_state(q0, v0)
        tq, tv = run.rollout(U, m.n_substeps, keep=True)
        out.append((tq, tv, run.status()))
    for k in (0, 1):
        a, b = out[0][k], out[1][k]
        assert np.abs(a - b).max() <= 1e-6 * max(np.abs(a).max(), 1.0), (k, np.abs(a - b).max())
    assert np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("order", ["in_order", "interleaved_sizes"])
def test_specialised_mixed_batch_matches_generic(order):
    """A mixed batch specialised per model (one kernel per model over its own blocks) against the
    generic kernel, every environment with its own model's substeps, 20 control steps."""
    import torch
    names = [("cartpole", 0, 70), ("quadruped", 1, 45), ("humanoid", 3, 33)]
    if order != "in_order":
        names = [names[1], names[2], names[0]]
    outs = []
    for spec in (False, True):
        parts = [(core.CompiledModel(W.model(nm)), n) for nm, _, n in names]
        batch = core.Batch(parts)
        if spec:
            batch.specialize(branch=False)
        st = core.State(batch, "cuda")
        ld = st.ld
        Q = np.zeros((batch.nq_max, ld), np.float32); V = np.zeros((batch.nv_max, ld), np.float32)
        U = np.zeros((20, max(batch.nu_max, 1), ld), np.float32)
        o = 0
        for (nm, cfg, n), (cm, _) in zip(names, parts):
            m = cm.src
            q0, v0 = W.initial_state(m, cfg, n)
            Q[:m.nq, o:o + n] = q0.T; V[:m.nv, o:o + n] = v0.T
            U[:, :m.nu, o:o + n] = W.actions(m, cfg, n, 0, 20).transpose(0, 2, 1)
            o += n
        st.qpos.copy_(torch.from_numpy(Q)); st.qvel.copy_(torch.from_numpy(V))
        ctrl = torch.from_numpy(U).to("cuda")
        for t in range(20):
            core.step(batch, st, ctrl[t], 0)
        torch.cuda.synchronize()
        outs.append((st.qpos.cpu().numpy(), st.qvel.cpu().numpy()))
    for a, b in zip(outs[0], outs[1]):
        assert np.allclose(a, b, rtol=1e-4, atol=1e-5)


def test_specialised_adjoint_matches_generic():
    """pg_step_vjp on a specialised batch (specialised forward, tape replay and reverse sweep)
    against the generic kernels: the same rollout gradient up to rounding."""
    import dataclasses
    from tests.test_gpu_adjoint import gpu_rollout_grad
    from oracle import oracle as O
    m = dataclasses.replace(W.quadruped(), iterations=100)
    q0, v0 = W.initial_state(m, 4, 8)
    U = W.actions(m, 4, 8, 0, 8)
    w = O.tracking_loss_weights(O.OracleModel(m))
    a = gpu_rollout_grad(m, q0, v0, U, w)
    b = gpu_rollout_grad(m, q0, v0, U, w, specialize=True)
    for k in ("q0", "v0", "u", "mass", "damping", "kp"):
        x, y = a[k], b[k]
        assert np.abs(x - y).max() <= 1e-4 * max(np.abs(x).max(), 1e-6), (k, np.abs(x - y).max())


@pytest.mark.parametrize("mname,spec", [("hand_elliptic", False), ("hand_elliptic", True), ("hand", True)])
def test_environments_per_warp_change_no_arithmetic(mname, spec):
    """8192 hands need more than one wave of blocks at 16 environments a warp, so the batch runs
    them 4 a warp (20 a block); a batch given 16 environments a block keeps 16 a warp.  The width
    only moves the workspaces: two control steps are bitwise equal."""
    m = W.model(mname)
    n = 8192
    q0, v0 = W.initial_state(m, 2, n)
    U = W.actions(m, 2, n, 0, 2)
    out = []
    for epc, width in ((0, 4), (16, 16)):
        run = GpuRun(m, n, envs_per_cta=epc)
        if spec:
            run.batch.specialize(branch=False)
        assert run.batch.kernel()["envs_per_warp"] == width
        run.set_state(q0, v0)
        run.rollout(U, m.n_substeps)
        out.append(run.get())
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
