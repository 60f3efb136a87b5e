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


def test_autotune_returns_a_working_shape(tmp_path, monkeypatch):
    monkeypatch.setattr(rollout, "_CACHE", str(tmp_path / "autotune.json"))
    parts = [(core.CompiledModel(W.quadruped()), 300), (core.CompiledModel(W.cartpole()), 200)]
    e = rollout.autotune(parts)
    assert e in rollout.candidate_shapes([m for m, _ in parts], [n for _, n in parts], 148)
    assert rollout.autotune(parts) == e           # cached
    # the tuned shape gives the same results as the default shape
    outs = []
    for epc in (0, e):
        b = core.Batch(parts, envs_per_cta=epc)
        st = core.State(b)
        q0, v0 = W.initial_state(W.quadruped(), 1, 300)
        st.qpos[:19, :300] = torch.from_numpy(q0.T).cuda()
        ctrl = torch.zeros((12, st.ld), device="cuda")
        ctrl[:, :300] = torch.from_numpy(W.actions(W.quadruped(), 1, 300, 0, 1)[0].T).cuda()
        core.step(b, st, ctrl, 0)
        outs.append(st.qpos[:, :300].cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
