"""Helpers shared by the GPU tests: run the CUDA path on env-major numpy inputs."""
from __future__ import annotations

import numpy as np
import torch

from paper_2502_08844_b300 import core
from paper_2502_08844_b300 import workloads as W


class GpuRun:
    def __init__(self, model: W.Model, n: int, envs_per_cta: int = 0, device="cuda", specialize=False):
        """specialize: False (the library's generic kernel), True (the model-specialised
        thread-per-environment kernel), "branch" (the branch-parallel kernel, which the model must
        qualify for, in its default launch: a barrier per substep) or "branch-warp" (the same
        kernel in blocks of one warp)."""
        self.model = model
        self.cm = core.CompiledModel(model)
        self.batch = core.Batch([(self.cm, n)], envs_per_cta=envs_per_cta)
        if specialize:
            branch = specialize in ("branch", "branch-warp")
            self.batch.specialize(branch=branch, warp_blocks=specialize == "branch-warp")
            if branch:
                k = self.batch.kernel()
                assert k["kernel"] == "branch-parallel" and k["barrier_per_substep"] == (specialize == "branch"), k
        self.state = core.State(self.batch, device)
        self.n = n
        self.device = device

    def set_state(self, qpos: np.ndarray, qvel: np.ndarray, warm: np.ndarray = None):
        ld = self.state.ld
        self.state.qpos.copy_(torch.from_numpy(core.to_soa(np.asarray(qpos, np.float32), ld, self.batch.nq_max)))
        self.state.qvel.copy_(torch.from_numpy(core.to_soa(np.asarray(qvel, np.float32), ld, self.batch.nv_max)))
        w = np.zeros_like(qvel, np.float32) if warm is None else np.asarray(warm, np.float32)
        self.state.qacc_warm.copy_(torch.from_numpy(core.to_soa(w, ld, self.batch.nv_max)))
        self.state.status.zero_()

    def ctrl_tensor(self, u: np.ndarray) -> torch.Tensor:
        """u [N, nu] -> device [nu_max, ld]"""
        return torch.from_numpy(core.to_soa(np.asarray(u, np.float32).reshape(self.n, -1), self.state.ld,
                                            max(self.batch.nu_max, 1))).to(self.device)

    def step(self, u: np.ndarray, n_substeps: int):
        core.step(self.batch, self.state, self.ctrl_tensor(u), n_substeps)

    def rollout(self, ctrl: np.ndarray, n_substeps: int, keep=False):
        traj_q, traj_v = [], []
        cts = [self.ctrl_tensor(ctrl[t]) for t in range(ctrl.shape[0])]
        for t in range(ctrl.shape[0]):
            core.step(self.batch, self.state, cts[t], n_substeps)
            if keep:
                q, v, _ = self.get()
                traj_q.append(q); traj_v.append(v)
        torch.cuda.synchronize()
        return (np.stack(traj_q), np.stack(traj_v)) if keep else None

    def get(self):
        torch.cuda.synchronize()
        n, m = self.n, self.model
        q = self.state.qpos[: m.nq, :n].cpu().numpy().T.astype(np.float64)
        v = self.state.qvel[: m.nv, :n].cpu().numpy().T.astype(np.float64)
        w = self.state.qacc_warm[: m.nv, :n].cpu().numpy().T.astype(np.float64)
        return q, v, w

    def status(self):
        torch.cuda.synchronize()
        return self.state.status.cpu().numpy().view(np.uint32)

    def debug(self, u: np.ndarray, env: int):
        return core.debug_substep(self.batch, self.state, self.ctrl_tensor(u), env)


def quat_canon(q: np.ndarray) -> np.ndarray:
    """Quaternion sign convention for comparisons (w >= 0)."""
    q = np.array(q, dtype=np.float64)
    s = np.where(q[..., :1] < 0, -1.0, 1.0)
    return q * s


def canon_qpos(model: W.Model, q: np.ndarray) -> np.ndarray:
    q = np.array(q, dtype=np.float64)
    adr = model.jnt_qposadr()
    for j, t in enumerate(model.jnt_type):
        if t == W.FREE:
            a = adr[j] + 3
            q[..., a:a + 4] = quat_canon(q[..., a:a + 4])
    return q


def rel_err(x, ref, atol=1e-6):
    """max over elements of |x - ref| / (|ref| + atol/rtol-scale) expressed as the smallest rtol
    such that |x - ref| <= rtol |ref| + atol holds."""
    x = np.asarray(x, np.float64); ref = np.asarray(ref, np.float64)
    d = np.abs(x - ref)
    over = d - atol
    if np.all(over <= 0):
        return 0.0
    return float(np.max(np.where(over > 0, over / np.maximum(np.abs(ref), 1e-300), 0.0)))


class MixedRun:
    """Several models in one batch (one launch per control step)."""

    def __init__(self, parts, envs_per_cta: int = 0, device="cuda", specialize: bool = False):
        self.parts = parts                      # [(workloads.Model, count)]
        self.cms = {}
        models = []
        for m, n in parts:
            if id(m) not in self.cms:
                self.cms[id(m)] = core.CompiledModel(m)
            models.append((self.cms[id(m)], n))
        self.batch = core.Batch(models, envs_per_cta=envs_per_cta)
        if specialize:   # True: thread-per-environment parts; "branch": branch-parallel parts where a model qualifies
            self.batch.specialize(branch=specialize == "branch")
        self.state = core.State(self.batch, device)
        self.offs = list(np.cumsum([0] + [n for _, n in parts]))
        self.n = self.offs[-1]
        self.device = device

    def set_state(self, qs, vs):
        ld = self.state.ld
        Q = np.zeros((self.batch.nq_max, ld), np.float32)
        V = np.zeros((self.batch.nv_max, ld), np.float32)
        for (m, n), o, q, v in zip(self.parts, self.offs, qs, vs):
            Q[:m.nq, o:o + n] = q.T
            V[:m.nv, o:o + n] = v.T
        self.state.qpos.copy_(torch.from_numpy(Q))
        self.state.qvel.copy_(torch.from_numpy(V))
        self.state.qacc_warm.zero_()
        self.state.status.zero_()

    def ctrl_tensor(self, us):
        U = np.zeros((max(self.batch.nu_max, 1), self.state.ld), np.float32)
        for (m, n), o, u in zip(self.parts, self.offs, us):
            U[:m.nu, o:o + n] = u.T
        return torch.from_numpy(U).to(self.device)

    def get(self):
        torch.cuda.synchronize()
        out = []
        for (m, n), o in zip(self.parts, self.offs):
            q = self.state.qpos[:m.nq, o:o + n].cpu().numpy().T.astype(np.float64)
            v = self.state.qvel[:m.nv, o:o + n].cpu().numpy().T.astype(np.float64)
            out.append((q, v))
        return out
