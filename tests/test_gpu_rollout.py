"""CUDA-graph rollouts and the launch-shape autotuner (GPU)."""
import numpy as np
import pytest
import torch

from paper_2502_08844_b300 import core, rollout
from paper_2502_08844_b300 import workloads as W
from tests.gpu_helpers import MixedRun

pytestmark = pytest.mark.gpu


def _mixed(T=20):
    parts = [("cartpole", 0, 50), ("quadruped", 1, 70), ("humanoid", 3, 30)]
    run = MixedRun([(W.model(nm), n) for nm, _, n in parts])
    qs, vs, us = [], [], []
    for nm, cfg, n in parts:
        m = W.model(nm)
        q, v = W.initial_state(m, cfg, n)
        qs.append(q); vs.append(v)
        us.append(W.actions(m, cfg, n, 0, T))
    ctrl = torch.stack([run.ctrl_tensor([u[t] for u in us]) for t in range(T)])
    return run, qs, vs, ctrl


def test_graph_replay_equals_eager_rollout():
    run, qs, vs, ctrl = _mixed()
    run.set_state(qs, vs)
    g = rollout.GraphRollout(run.batch, run.state, ctrl, 0)
    g.run_eager()
    eager = [(q.copy(), v.copy()) for q, v in run.get()]
    run.set_state(qs, vs)
    g.capture()          # capture does not execute the steps
    run.set_state(qs, vs)
    g.replay()
    replay = run.get()
    for (qa, va), (qb, vb) in zip(eager, replay):
        assert np.array_equal(qa, qb) and np.array_equal(va, vb)


def test_autotune_returns_a_working_choice(tmp_path, monkeypatch):
    """The autotuner's (kernel, envs per block) is one of its candidates, is cached, and its batch
    steps as the generic kernel's does (to rounding: the kernels order their arithmetic
    differently; bitwise where it picked the generic kernel)."""
    monkeypatch.setattr(rollout, "_CACHE", str(tmp_path / "autotune.json"))
    parts = [(core.CompiledModel(W.quadruped()), 300), (core.CompiledModel(W.cartpole()), 200)]
    choice = rollout.autotune(parts)
    models, counts = [m for m, _ in parts], [n for _, n in parts]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert choice in rollout.candidates(models, counts, sms)
    assert rollout.autotune(parts) == choice           # cached
    assert ("branch", 0) in rollout.candidates(models, counts, sms)   # the quadruped qualifies
    outs = []
    for b in (core.Batch(parts), rollout.make_batch(parts, choice)):
        st = core.State(b)
        q0, v0 = W.initial_state(W.quadruped(), 1, 300)
        st.qpos[:19, :300] = torch.from_numpy(q0.T).cuda()
        ctrl = torch.zeros((12, st.ld), device="cuda")
        ctrl[:, :300] = torch.from_numpy(W.actions(W.quadruped(), 1, 300, 0, 1)[0].T).cuda()
        core.step(b, st, ctrl, 0)
        outs.append(st.qpos[:, :300].cpu().numpy())
    if choice[0] == "generic":
        assert np.array_equal(outs[0], outs[1])
    else:
        np.testing.assert_allclose(outs[1], outs[0], rtol=1e-5, atol=1e-6)


def test_autotune_generic_only_and_shapes():
    """The kernel list restricts the search; the shapes fit shared memory and 8 warps."""
    parts = [(core.CompiledModel(W.humanoid()), 100)]
    models = [m for m, _ in parts]
    shapes = rollout.candidate_shapes(models, [100], 148)
    ws = models[0].sizes.workspace_bytes
    assert shapes[0] == 0 and all(16 <= e <= 256 and e * ws <= rollout.SMEM_PER_BLOCK for e in shapes[1:])
    assert all(k == "generic" for k, _ in rollout.candidates(models, [100], 148, ("generic",)))


def _host_case(specialize, n=300, T=7):
    m = W.quadruped()
    outs = []
    for pipelined in (False, True):
        b = core.Batch([(core.CompiledModel(m), n)])
        if specialize:
            b.specialize()
        st = core.State(b)
        q0, v0 = W.initial_state(m, 1, n)
        st.qpos.copy_(torch.from_numpy(core.to_soa(q0, st.ld, b.nq_max)))
        st.qvel.copy_(torch.from_numpy(core.to_soa(v0, st.ld, b.nv_max)))
        U = np.stack([core.to_soa(u, st.ld, b.nu_max) for u in W.actions(m, 1, n, 0, T)])
        ctrl_h = torch.from_numpy(U).pin_memory()
        qh = torch.zeros((T, b.nq_max, st.ld)).pin_memory()
        vh = torch.zeros((T, b.nv_max, st.ld)).pin_memory()
        if pipelined:
            core.rollout_host(b, st, ctrl_h, qh, vh, m.n_substeps)
        else:
            for t in range(T):
                core.step_host(b, st, ctrl_h[t], qh[t], vh[t], m.n_substeps)
        torch.cuda.synchronize()
        outs.append((qh.numpy().copy(), vh.numpy().copy(), st.qpos.cpu().numpy(), st.qvel.cpu().numpy()))
    return outs


@pytest.mark.parametrize("specialize", [pytest.param(False, id="generic"), pytest.param(True, id="branch")])
def test_rollout_host_equals_step_host_per_step(specialize):
    """pg_rollout_host (uploads, steps and downloads overlapped on three streams) returns every
    step's state bitwise equal to pg_step_host called once per step, and leaves the same state"""
    (qa, va, qda, vda), (qb, vb, qdb, vdb) = _host_case(specialize)
    assert np.array_equal(qa, qb) and np.array_equal(va, vb)
    assert np.array_equal(qda, qdb) and np.array_equal(vda, vdb)
    assert np.isfinite(qb).all() and not np.array_equal(qb[0], qb[-1])


def test_rollout_host_twice_and_zero_steps():
    """two rollouts back to back reuse the staging buffers in order; 0 steps does nothing; NULL
    host buffers are refused"""
    from paper_2502_08844_b300 import _capi
    m = W.quadruped()
    n, T = 64, 5
    b = core.Batch([(core.CompiledModel(m), n)])
    st = core.State(b)
    q0, v0 = W.initial_state(m, 1, n)
    st.qpos.copy_(torch.from_numpy(core.to_soa(q0, st.ld, b.nq_max)))
    st.qvel.copy_(torch.from_numpy(core.to_soa(v0, st.ld, b.nv_max)))
    U = np.stack([core.to_soa(u, st.ld, b.nu_max) for u in W.actions(m, 1, n, 0, 2 * T)])
    ctrl_h = torch.from_numpy(U).pin_memory()
    qh = torch.zeros((2 * T, b.nq_max, st.ld)).pin_memory()
    vh = torch.zeros((2 * T, b.nv_max, st.ld)).pin_memory()
    core.rollout_host(b, st, ctrl_h[:T], qh[:T], vh[:T], m.n_substeps)
    core.rollout_host(b, st, ctrl_h[T:], qh[T:], vh[T:], m.n_substeps)
    core.rollout_host(b, st, ctrl_h[:0], qh[:0], vh[:0], m.n_substeps)
    torch.cuda.synchronize()
    ref = core.State(b)
    ref.qpos.copy_(torch.from_numpy(core.to_soa(q0, st.ld, b.nq_max)))
    ref.qvel.copy_(torch.from_numpy(core.to_soa(v0, st.ld, b.nv_max)))
    for t in range(2 * T):
        core.step(b, ref, ctrl_h[t].cuda(), m.n_substeps)
        torch.cuda.synchronize()
        assert np.array_equal(ref.qpos.cpu().numpy(), qh[t].numpy())
    with pytest.raises(_capi.PgError):
        _capi.pg_rollout_host(b.handle, st.c(), ctrl_h.data_ptr(), None, vh.data_ptr(), 1, 0, None)


def test_rollout_host_staging_grows_for_a_wider_state():
    """a rollout on a state of larger row pitch right after one on the batch's own state (still
    queued, not synchronised) regrows the staging buffers; both rollouts return every step's state
    bitwise equal to pg_step on a reference state"""
    m = W.quadruped()
    n, T = 64, 4
    b = core.Batch([(core.CompiledModel(m), n)])
    q0, v0 = W.initial_state(m, 1, n)
    U = W.actions(m, 1, n, 0, T)

    def state(ld):
        st = core.State(b)
        st.ld = ld
        st.qpos = torch.from_numpy(core.to_soa(q0, ld, b.nq_max)).cuda()
        st.qvel = torch.from_numpy(core.to_soa(v0, ld, b.nv_max)).cuda()
        st.qacc_warm = torch.zeros((b.nv_max, ld), dtype=torch.float32, device="cuda")
        return st

    runs = []
    for ld in (core.State(b).ld, core.State(b).ld + 96):
        st = state(ld)
        ctrl_h = torch.from_numpy(np.stack([core.to_soa(u, ld, b.nu_max) for u in U])).pin_memory()
        qh = torch.zeros((T, b.nq_max, ld)).pin_memory()
        vh = torch.zeros((T, b.nv_max, ld)).pin_memory()
        core.rollout_host(b, st, ctrl_h, qh, vh, m.n_substeps)   # the second call regrows
        runs.append((ld, ctrl_h, qh, vh))
    torch.cuda.synchronize()
    for ld, ctrl_h, qh, vh in runs:
        ref = state(ld)
        for t in range(T):
            core.step(b, ref, ctrl_h[t].cuda(), m.n_substeps)
            torch.cuda.synchronize()
            assert np.array_equal(ref.qpos.cpu().numpy()[:, :n], qh[t].numpy()[:, :n]), (ld, t)
            assert np.array_equal(ref.qvel.cpu().numpy()[:, :n], vh[t].numpy()[:, :n]), (ld, t)
