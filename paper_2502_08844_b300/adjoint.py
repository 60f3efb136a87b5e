"""Differentiable rollouts: the hand-written CUDA adjoint (pg_step_vjp) behind torch.autograd.

`rollout(batch, qpos0, qvel0, ctrl, params)` runs T control steps with pg_step and returns the
trajectories. Their gradients flow back to:

* the initial state;
* every control;
* the per-environment model parameters: body masses, dof damping and actuator kp.

The forward pass keeps a checkpoint of the state (qpos, qvel and the solver's warm start) every
`segment` control steps; that is all the backward pass keeps of the forward. The backward pass
replays each segment from its checkpoint on the GPU, last segment first, recording each
substep's start state. It then sweeps the segment's steps back with the CUDA adjoint kernel.

The contact solve is differentiated implicitly at the solver's final iterate. The gradient is
exact when the solver has converged, i.e. when its iteration cap is not hit.
"""
from __future__ import annotations

from typing import Optional, Tuple

import torch

from . import _capi, core


class PgRollout(torch.autograd.Function):
    """(qpos0 [nq_max, ld], qvel0 [nv_max, ld], ctrl [T, nu_max, ld], params [nparam_max, ld]) ->
    (qpos [T, nq_max, ld], qvel [T, nv_max, ld]): the state after each control step.

    `params` carries no values into the step: the model's compiled masses, damping and kp are
    used. It is the tensor that receives their per-environment gradient (rows: body masses |
    dof damping | actuator kp of the environment's model, see `param_values`)."""

    @staticmethod
    def forward(ctx, qpos0, qvel0, ctrl, params, batch: core.Batch, n_substeps: int, segment: int):
        # the backward sweep's scratch, reserved here so that the backward pass allocates nothing
        _capi.pg_batch_reserve_vjp(batch.handle, min(segment, ctrl.shape[0]), n_substeps, ctrl.shape[-1])
        st = core.State(batch, qpos0.device)
        st.qpos.copy_(qpos0)
        st.qvel.copy_(qvel0)
        T = ctrl.shape[0]
        Q = torch.empty((T,) + tuple(st.qpos.shape), dtype=torch.float32, device=qpos0.device)
        V = torch.empty((T,) + tuple(st.qvel.shape), dtype=torch.float32, device=qpos0.device)
        ckpts = []
        for t in range(T):
            if t % segment == 0:
                ckpts += [st.qpos.clone(), st.qvel.clone(), st.qacc_warm.clone()]
            core.step(batch, st, ctrl[t], n_substeps)
            Q[t].copy_(st.qpos)
            V[t].copy_(st.qvel)
        ctx.batch, ctx.n_substeps, ctx.segment, ctx.T = batch, n_substeps, segment, T
        ctx.save_for_backward(ctrl, *ckpts)
        return Q, V

    @staticmethod
    def backward(ctx, gQ: Optional[torch.Tensor], gV: Optional[torch.Tensor]):
        batch, seg, T = ctx.batch, ctx.segment, ctx.T
        ctrl, *ck = ctx.saved_tensors
        dev = ctrl.device
        ld = ctrl.shape[-1]
        adj_q = torch.zeros((batch.nq_max, ld), dtype=torch.float32, device=dev)
        adj_v = torch.zeros((batch.nv_max, ld), dtype=torch.float32, device=dev)
        g_ctrl = torch.zeros_like(ctrl)
        g_par = torch.zeros((batch.nparam_max, ld), dtype=torch.float32, device=dev)
        st = core.State(batch, dev)
        gQ = None if gQ is None else gQ.contiguous()
        gV = None if gV is None else gV.contiguous()
        for k in reversed(range((T + seg - 1) // seg)):
            t0, t1 = k * seg, min(T, (k + 1) * seg)
            st.qpos, st.qvel, st.qacc_warm = ck[3 * k], ck[3 * k + 1], ck[3 * k + 2]
            core.step_vjp(batch, st, ctrl[t0:t1], ctx.n_substeps, None if gQ is None else gQ[t0:t1],
                          None if gV is None else gV[t0:t1], adj_q, adj_v, g_ctrl[t0:t1], g_par)
        return adj_q, adj_v, g_ctrl, g_par, None, None, None


def param_values(batch: core.Batch, ld: int, device="cuda") -> torch.Tensor:
    """[nparam_max, ld] tensor of each environment's model parameters (body masses | dof damping |
    actuator kp), the layout of PgRollout's `params` and of its gradient."""
    import numpy as np
    out = np.zeros((batch.nparam_max, ld), np.float32)
    for m, o, n in zip(batch.models, batch.env_off, batch.counts):
        src = m.src
        vals = np.concatenate([src.body_mass, src.dof_damping, src.act_kp]).astype(np.float32)
        out[:len(vals), o:o + n] = vals[:, None]
    return torch.from_numpy(out).to(device)


def rollout(batch: core.Batch, qpos0: torch.Tensor, qvel0: torch.Tensor, ctrl: torch.Tensor,
            params: Optional[torch.Tensor] = None, n_substeps: int = 0, segment: int = 8) -> Tuple[torch.Tensor, torch.Tensor]:
    """Differentiable T-step rollout (see PgRollout); params defaults to param_values(batch)."""
    if params is None:
        params = param_values(batch, ctrl.shape[-1], ctrl.device)
    return PgRollout.apply(qpos0, qvel0, ctrl, params, batch, n_substeps, segment)
