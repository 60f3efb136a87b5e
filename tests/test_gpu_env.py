"""GPU parity of the locomotion task around the step (pg_env_reset / pg_env_step) against the
FP64 oracle (oracle/env.py), through the C ABI.

Tolerances: the physics inside the step is held to the one-step bound (1e-5 relative to the
largest state entry, 1e-6 absolute); observations are rotations and differences of that state,
so they get 2e-5 of the state's scale.  Reward terms are sums and exponentials of squared
state quantities. The PD torque multiplies the joint error by kp = 35 and the torque term
squares it, so a 1e-5 state error reaches ~1e-4 of the term: terms are compared at 1e-3
relative. The clearance term's fourth root of a foot's squared speed turns a 1e-5 speed error
at rest into ~3e-3 of the root, so the absolute floor is 1e-4.  The integer
decisions (done, truncated, the feet's contact flags) must match exactly, except a contact flag
whose foot lies within 5e-5 m of the contact height (float32 rounding of the state can move a
foot across it); environments with such a foot are left out of the contact-dependent checks.
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

from paper_2502_08844_b300 import core, workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _oracle():
    from oracle import env as E
    from oracle import oracle as O
    return O, E


def _quat_axis(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * a])


class Setup:
    """A quadruped batch with its task, states and task states (float32, env-major host copies)."""

    def __init__(self, n, task, specialize=False, seed=0):
        self.m = W.quadruped()
        self.task = task
        self.cm = core.CompiledModel(self.m)
        self.batch = core.Batch([(self.cm, n)])
        if specialize:
            self.batch.specialize()
        self.t = core.Task(self.cm, task)
        self.state = core.State(self.batch, DEV)
        self.n, self.ld = n, self.state.ld
        rng = np.random.default_rng(seed)
        m = self.m
        q, v = W.initial_state(m, 1, n, noise=0.04)
        q[:, 2] += rng.uniform(-0.004, 0.03, n).astype(np.float32)   # some feet down, some up
        self.q = q; self.v = v
        self.q0, self.v0 = W.initial_state(m, 1, n, env0=10_000, noise=0.02)
        self.cmd = W.commands(1, n)
        self.U = W.policy_actions(m, 1, n, 0, 16)
        nu, nf = m.nu, task.nfeet
        st = np.zeros((n, 2 * nu + 2 * nf + 1), np.float32)
        st[:, :nu] = task.q_default + rng.uniform(-0.2, 0.2, (n, nu))
        st[:, nu:2 * nu] = rng.uniform(-1, 1, (n, nu))
        st[:, 2 * nu:2 * nu + nf] = rng.uniform(0.0, 0.4, (n, nf))
        st[:, 2 * nu + nf:2 * nu + 2 * nf] = rng.integers(0, 2, (n, nf))
        st[:, -1] = rng.integers(0, 8, n)
        self.task_state = st

    def upload(self):
        ld, s = self.ld, self.state
        dev = lambda a, rows: torch.from_numpy(core.to_soa(a, ld, rows)).to(DEV)
        s.qpos.copy_(dev(self.q, self.batch.nq_max)); s.qvel.copy_(dev(self.v, self.batch.nv_max))
        s.qacc_warm.zero_(); s.status.zero_()
        self.d_task_state = dev(self.task_state, self.t.state_rows)
        self.d_q0 = dev(self.q0, self.batch.nq_max); self.d_v0 = dev(self.v0, self.batch.nv_max)
        self.d_cmd = dev(self.cmd, 3)
        self.obs = torch.zeros((self.t.nobs, ld), device=DEV)
        self.rew = torch.zeros(ld, device=DEV); self.done = torch.zeros(ld, device=DEV)
        self.trunc = torch.zeros(ld, device=DEV)
        self.terms = torch.zeros((self.t.nterms, ld), device=DEV)

    def step(self, k, n_substeps=5):
        a = torch.from_numpy(core.to_soa(self.U[k], self.ld, self.m.nu)).to(DEV)
        core.env_step(self.batch, self.t, self.state, self.d_task_state, a, self.d_cmd, self.d_q0, self.d_v0,
                      n_substeps, self.obs, self.rew, self.done, self.trunc, self.terms)
        torch.cuda.synchronize()

    def host(self):
        n = self.n
        T = lambda x: x[:, :n].cpu().numpy().T.astype(np.float64)
        s = self.state
        return dict(qpos=T(s.qpos[:self.m.nq]), qvel=T(s.qvel[:self.m.nv]), warm=T(s.qacc_warm[:self.m.nv]),
                    task_state=T(self.d_task_state), obs=T(self.obs), terms=T(self.terms),
                    reward=self.rew[:n].cpu().numpy().astype(np.float64), done=self.done[:n].cpu().numpy(),
                    truncated=self.trunc[:n].cpu().numpy(), status=s.status[:n].cpu().numpy())


def _near_contact(ot, qpos, qvel, h):
    _, height, _ = ot.feet(qpos, qvel)
    return np.any(np.abs(height - h) < 5e-5)


def _compare_env(ot, g, e, pre, a, cmd, q0, v0, warm, tol_terms=1e-3):
    """GPU results g (host dict, env e) against the oracle's step from the GPU's pre-step state."""
    o = ot.step(pre["qpos"][e], pre["qvel"][e], warm, pre["task_state"][e], a, cmd, q0, v0, 5)
    assert g["done"][e] == o["done"] and g["truncated"][e] == o["truncated"], e
    near = _near_contact(ot, o["qpos_final"], o["qvel_final"], ot.contact_height)
    nu, nf = ot.nu, ot.nf
    if o["done"]:
        assert np.array_equal(g["qpos"][e], np.asarray(q0, np.float32).astype(np.float64)), e
        assert np.array_equal(g["qvel"][e], np.asarray(v0, np.float32).astype(np.float64)), e
        assert np.all(g["warm"][e] == 0) and g["status"][e] == 0
        assert np.array_equal(g["task_state"][e], ot.initial_task_state().astype(np.float32).astype(np.float64))
    else:
        for k in ("qpos", "qvel"):
            err = max(np.abs(g[k][e] - o[k]).max() - 1e-6, 0.0) / np.abs(o[k]).max()
            assert err <= 1e-5, (e, k, err)
        gs, os_ = g["task_state"][e], o["task_state"]
        assert np.allclose(gs[:2 * nu], os_[:2 * nu], atol=2e-6), e       # q_des, previous action
        assert gs[-1] == os_[-1], e                                        # episode step
        if not near:
            assert np.array_equal(gs[2 * nu + nf:2 * nu + 2 * nf], os_[2 * nu + nf:2 * nu + 2 * nf]), e
            assert np.allclose(gs[2 * nu:2 * nu + nf], os_[2 * nu:2 * nu + nf], atol=1e-6), e
    scale = max(1.0, np.abs(o["qvel"]).max(), np.abs(o["qpos"]).max())
    assert np.abs(g["obs"][e] - o["obs"]).max() <= 2e-5 * scale + 2e-6, (e, np.abs(g["obs"][e] - o["obs"]).max())
    if not near:
        d = np.abs(g["terms"][e] - o["terms"])
        bad = d > tol_terms * np.abs(o["terms"]) + 1e-4
        assert not bad.any(), (e, [W.TERMS[i] for i in np.nonzero(bad)[0]], g["terms"][e][bad], o["terms"][bad])
        assert abs(g["reward"][e] - o["reward"]) <= tol_terms * (abs(o["reward"]) + np.abs(ot.weight * o["terms"]).sum()) + 1e-4
    return near


@pytest.mark.parametrize("specialize", [pytest.param(False, id="generic"), pytest.param(True, id="branch")])
@pytest.mark.parametrize("mode", [W.ABSOLUTE, W.RELATIVE])
def test_env_step_matches_oracle(mode, specialize):
    """One environment step of 200 quadrupeds (a ragged last warp): some upright, some turned
    over (terminated), some at the end of their episode (truncated).  With specialisation the
    step runs as three launches: the joint targets, the substeps on the branch-parallel kernel
    and the step's end (reward to observation)."""
    O, E = _oracle()
    task = dataclasses.replace(W.quadruped_task(action_mode=mode), episode_length=8)
    S = Setup(200, task, specialize=specialize)
    if specialize:
        assert S.batch.kernel()["kernel"] == "branch-parallel"
    S.q[::17, 2] += 0.3
    S.q[::17, 3:7] = _quat_axis((1, 0, 0), math.pi * 0.95).astype(np.float32)   # turned over
    S.task_state[5::23, -1] = 7                                                    # last step of the episode
    S.upload()
    pre = dict(qpos=S.q.astype(np.float64), qvel=S.v.astype(np.float64), task_state=S.task_state.astype(np.float64))
    S.step(0)
    g = S.host()
    ot = E.OracleTask(O.OracleModel(S.m), task)
    assert g["done"][::17].all() and not g["truncated"][::17].any()
    assert g["truncated"][5::23][[i for i in range(len(g["truncated"][5::23])) if (5 + 23 * i) % 17]].all()
    assert 0 < g["done"].sum() < S.n
    skipped = 0
    for e in range(S.n):
        skipped += _compare_env(ot, g, e, pre, S.U[0][e], S.cmd[e], S.q0[e], S.v0[e], np.zeros(S.m.nv))
    assert skipped < S.n // 4


@pytest.mark.parametrize("specialize", [pytest.param(False, id="generic"), pytest.param(True, id="branch")])
def test_env_rollout_with_resets_matches_oracle_step_by_step(specialize):
    """12 environment steps with 5-step episodes: every environment restarts twice.  Each step
    is checked against the oracle's step from the GPU's own pre-step state and warm start."""
    O, E = _oracle()
    task = W.quadruped_task(episode_length=5)
    S = Setup(64, task, specialize=specialize, seed=1)
    S.task_state[:, -1] = 0
    S.upload()
    ot = E.OracleTask(O.OracleModel(S.m), task)
    dones = np.zeros(S.n)
    for k in range(12):
        pre = S.host()
        S.step(k)
        g = S.host()
        for e in range(0, S.n, 3):
            _compare_env(ot, g, e, pre, S.U[k][e], S.cmd[e], S.q0[e], S.v0[e], pre["warm"][e])
        dones += g["done"]
    assert np.all(dones == 2)


def test_env_reset_matches_oracle():
    O, E = _oracle()
    task = W.quadruped_task()
    S = Setup(100, task, seed=2)
    S.upload()
    core.env_reset(S.batch, S.t, S.state, S.d_task_state, S.d_q0, S.d_v0, S.d_cmd, S.obs)
    torch.cuda.synchronize()
    g = S.host()
    ot = E.OracleTask(O.OracleModel(S.m), task)
    for e in range(S.n):
        q, v, w, st, obs = ot.reset(S.q0[e], S.v0[e], S.cmd[e])
        assert np.array_equal(g["qpos"][e], q) and np.array_equal(g["qvel"][e], v) and np.all(g["warm"][e] == 0)
        assert np.array_equal(g["task_state"][e], st.astype(np.float32).astype(np.float64))
        assert np.abs(g["obs"][e] - obs).max() <= 2e-6


def test_specialised_env_step_matches_generic():
    task = W.quadruped_task(episode_length=6)
    outs = []
    for spec in (False, True):
        S = Setup(256, task, specialize=spec, seed=3)
        S.upload()
        for k in range(8):
            S.step(k)
        outs.append(S.host())
    a, b = outs
    for k in ("done", "truncated"):
        assert np.array_equal(a[k], b[k])
    for k in ("qpos", "qvel", "obs", "terms", "reward", "task_state"):
        assert np.allclose(a[k], b[k], rtol=1e-4, atol=1e-5), k


def test_env_step_argument_errors():
    from paper_2502_08844_b300 import _capi
    task = W.quadruped_task()
    S = Setup(8, task)
    S.upload()
    other = core.Batch([(core.CompiledModel(W.quadruped()), 8)])
    with pytest.raises(_capi.PgError) as ei:
        core.env_reset(other, S.t, core.State(other, DEV), S.d_task_state, S.d_q0, S.d_v0, S.d_cmd, S.obs)
    assert ei.value.code == _capi.PG_EUNSUPPORTED
    rc = _capi._lib.pg_env_step(S.batch.handle, S.t.handle, S.state.c(), None, None, None, None, None, 5,
                                None, None, None, None, None, None, None)
    assert rc == _capi.PG_EINVAL


def test_env_step_with_per_environment_parameters():
    """pg_env_step with a per-environment parameter block: each environment against the oracle's
    task on its substituted model (oracle.randomize), calibration offsets and PD gain scales (in
    the physics and in the reward's PD torques) included."""
    O, E = _oracle()
    from oracle import randomize as RZ
    task = W.quadruped_task(episode_length=50)
    S = Setup(24, task, seed=4)
    S.task_state[:, -1] = 0
    S.upload()
    P = W.randomized_params(S.m, 1, S.n)
    params = torch.from_numpy(core.to_soa(P, S.ld, P.shape[1])).to(DEV)
    a = torch.from_numpy(core.to_soa(S.U[0], S.ld, S.m.nu)).to(DEV)
    core.env_step(S.batch, S.t, S.state, S.d_task_state, a, S.d_cmd, S.d_q0, S.d_v0, 5, S.obs, S.rew, S.done,
                  S.trunc, S.terms, params=params)
    torch.cuda.synchronize()
    g = S.host()
    pre = dict(qpos=S.q.astype(np.float64), qvel=S.v.astype(np.float64), task_state=S.task_state.astype(np.float64))
    nb, nv = S.m.nbody, S.m.nv
    for e in range(S.n):
        ot = E.OracleTask(O.OracleModel(RZ.substituted_model(S.m, P[e])), task)
        r = RZ.rows(S.m)["calibration"]
        ot.calibration = P[e, r:r + S.m.nu].astype(np.float64)
        _compare_env(ot, g, e, pre, S.U[0][e], S.cmd[e], S.q0[e], S.v0[e], np.zeros(nv))
