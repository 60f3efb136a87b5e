"""Torch-facing wrapper of the C ABI: compiled models, batches, batch state and the step.

PyTorch only provides device memory and streams here; every step of the physics runs in
the CUDA library (`libpg.so`) behind `_capi`.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import _capi
from . import workloads as W

_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int)


def _stream_ptr(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


class CompiledModel:
    """A model compiled by pg_model_compile from a workloads.Model description."""

    def __init__(self, m: W.Model):
        self.src = m
        keep = []

        def f(a):
            a = np.ascontiguousarray(np.asarray(a, np.float32))
            keep.append(a)
            return a.ctypes.data_as(_fp)

        def i(a):
            a = np.ascontiguousarray(np.asarray(a, np.int32))
            keep.append(a)
            return a.ctypes.data_as(_ip)

        pair_geom = m.pair_geom if m.npair else np.zeros((0, 2), np.int32)
        d = _capi.pg_model_desc(
            m.nbody, m.njnt, m.ngeom, m.npair, m.nu,
            i(m.body_parent), f(m.body_pos), f(m.body_quat), f(m.body_mass), f(m.body_ipos), f(m.body_inertia),
            i(m.body_geom_inertia), i(m.jnt_type), i(m.jnt_body), f(m.jnt_pos), f(m.jnt_axis), i(m.jnt_limited),
            f(m.jnt_range), f(m.dof_damping), f(m.dof_armature), f(m.dof_rotor), i(m.geom_type), i(m.geom_body),
            f(m.geom_pos), f(m.geom_quat), f(m.geom_size), f(m.geom_mass), i(pair_geom), f(m.pair_friction),
            i(m.pair_condim), i(m.act_type), i(m.act_jnt), f(m.act_gear), f(m.act_kp), f(m.act_kd),
            i(m.act_ctrllimited), f(m.act_ctrlrange), float(m.timestep), f(m.gravity), int(m.iterations),
            int(m.cone), float(m.impratio), f(m.solref), f(m.solimp), float(m.margin), int(m.max_contacts),
            int(m.n_substeps),
            0 if m.hfield is None else int(m.hfield.shape[0]), 0 if m.hfield is None else int(m.hfield.shape[1]),
            None if m.hfield is None else f(m.hfield),
            None if m.act_forcelimited is None else i(m.act_forcelimited),
            None if m.act_forcerange is None else f(m.act_forcerange),
            None if m.dof_frictionloss is None else f(m.dof_frictionloss),
            m.nmesh, *((i(m.mesh_vertadr), i(m.mesh_vertnum), f(m.mesh_vert), i(m.mesh_faceadr), i(m.mesh_facenum),
                        i(m.mesh_face), i(m.geom_meshid)) if m.nmesh else (None,) * 7))
        self.handle = _capi.pg_model_compile(d)
        self.sizes = _capi.pg_model_info(self.handle)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            _capi.pg_model_free(h)
            self.handle = None

    def branch_plan(self) -> dict:
        """pg_model_branch_plan: whether the model qualifies for the branch-parallel kernel."""
        k = _capi.pg_model_branch_plan(self.handle)
        return {"branch": k.kernel == _capi.PG_KERNEL_BRANCH, "lanes_per_env": k.lanes_per_env,
                "branches": k.branches, "reason": k.reason.decode()}

    def precompile(self, count: int, envs_per_cta: int = 0, branch: bool = True, cache_dir: str = None,
                   sms: int = 0) -> int:
        """pg_model_precompile: compile with NVRTC, without device work, the kernels that
        Batch.specialize(branch) needs for `count` environments of this model (a batch with
        envs_per_cta), into cache_dir (None: the disk cache).  Returns the thread-per-environment
        kernels' width."""
        return _capi.pg_model_precompile(self.handle, count, envs_per_cta, sms,
                                         _capi.PG_SPEC_BRANCH if branch else 0, cache_dir)

    def envs_per_warp(self, count: int, envs_per_cta: int = 0, sms: int = 0) -> int:
        """The thread-per-environment kernels' width (environments per warp) for `count`
        environments of this model, as pg_batch_compile chooses it (host only)."""
        return _capi.pg_model_precompile(self.handle, count, envs_per_cta, sms, _capi.PG_PRECOMPILE_WIDTH_ONLY, None)

    @property
    def nq(self):
        return self.sizes.nq

    @property
    def nv(self):
        return self.sizes.nv

    @property
    def nu(self):
        return self.sizes.nu


class Batch:
    """counts[k] consecutive environments of models[k], stepped in one launch."""

    def __init__(self, parts: Sequence[Tuple[CompiledModel, int]], envs_per_cta: int = 0):
        self.models = [m for m, _ in parts]
        self.counts = [int(c) for _, c in parts]
        self.handle = _capi.pg_batch_compile([m.handle for m in self.models], self.counts, envs_per_cta)
        self.n, self.nq_max, self.nv_max, self.nu_max = _capi.pg_batch_info(self.handle)
        self.env_off = list(np.cumsum([0] + self.counts[:-1]))
        # rows of the per-environment parameter gradient of pg_step_vjp (masses | damping | kp)
        self.nparam_max = max(m.sizes.nparam for m in self.models)
        self.specialized = False

    def specialize(self, branch: bool = True, warp_blocks: bool = False) -> None:
        """pg_batch_specialize_ex: compile (NVRTC, cached) step kernels specialised to the model;
        branch: let pg_step run the branch-parallel kernel when the model qualifies; warp_blocks:
        launch it in blocks of one warp without the per-substep barrier (PG_SPEC_BRANCH_WARP)."""
        flags = (_capi.PG_SPEC_BRANCH if branch else 0) | (_capi.PG_SPEC_BRANCH_WARP if warp_blocks else 0)
        _capi.pg_batch_specialize_ex(self.handle, flags)
        self.specialized = True

    def kernel(self) -> dict:
        """pg_batch_kernel: the kernel pg_step runs (name, lanes per environment, branches, and why
        the branch-parallel kernel is not used)."""
        k = _capi.pg_batch_kernel(self.handle)
        return {"kernel": _capi.KERNEL_NAMES[k.kernel], "lanes_per_env": k.lanes_per_env, "branches": k.branches,
                "reason": k.reason.decode(), "branch_parts": k.branch_parts, "barrier_per_substep": bool(k.sync),
                "branch_dr": bool(k.branch_dr), "branch_tape": bool(k.branch_tape), "envs_per_warp": k.envs_per_warp}

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            _capi.pg_batch_free(h)
            self.handle = None


class State:
    """Batch state in device memory: [coord][ld] float32 arrays, status [n] (uint32 bits)."""

    def __init__(self, batch: Batch, device="cuda"):
        self.n = batch.n
        self.ld = max(4, (batch.n + 3) // 4 * 4)
        self.qpos = torch.zeros((batch.nq_max, self.ld), dtype=torch.float32, device=device)
        self.qvel = torch.zeros((batch.nv_max, self.ld), dtype=torch.float32, device=device)
        self.qacc_warm = torch.zeros((batch.nv_max, self.ld), dtype=torch.float32, device=device)
        self.status = torch.zeros((self.n,), dtype=torch.int32, device=device)
        self.stats = None   # optional [3, ld] int32 solver counters (enable_stats)

    def enable_stats(self):
        self.stats = torch.zeros((3, self.ld), dtype=torch.int32, device=self.qpos.device)
        return self.stats

    def c(self) -> _capi.pg_state:
        return _capi.pg_state(self.qpos.data_ptr(), self.qvel.data_ptr(), self.qacc_warm.data_ptr(),
                              self.status.data_ptr(), self.n, self.ld,
                              None if self.stats is None else self.stats.data_ptr())


class Task:
    """A locomotion task (pg_task_compile) around a compiled model's step: the action mapping,
    the feet and the reward table's weights of a workloads.Task."""

    def __init__(self, model: CompiledModel, task: W.Task):
        self.model, self.src = model, task
        self._q_default = np.ascontiguousarray(task.q_default, np.float32)
        self._feet = np.ascontiguousarray(task.foot_geom, np.int32)
        w = (C.c_float * _capi.PG_NTERMS)(*[float(x) for x in task.weight])
        d = _capi.pg_task_desc(int(task.action_mode), float(task.action_scale),
                               self._q_default.ctypes.data_as(C.c_void_p), int(task.nfeet),
                               self._feet.ctypes.data_as(C.c_void_p), float(task.contact_height),
                               float(task.clearance_height), float(task.sigma_lin_vel), float(task.sigma_ang_vel),
                               float(task.air_time_min), float(task.air_time_max), w, int(task.episode_length))
        self.handle = _capi.pg_task_compile(model.handle, d)
        s = _capi.pg_task_info(self.handle)
        self.nobs, self.nterms, self.state_rows = s.nobs, s.nterms, s.state_rows

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            _capi.pg_task_free(h)
            self.handle = None


def env_reset(batch: Batch, task: Task, state: State, task_state: torch.Tensor, qpos0: torch.Tensor,
              qvel0: torch.Tensor, cmd: torch.Tensor, obs: torch.Tensor, stream=None) -> None:
    """pg_env_reset: every environment starts an episode at (qpos0, qvel0); obs is written."""
    ld = state.ld
    assert task_state.shape == (task.state_rows, ld) and obs.shape == (task.nobs, ld) and cmd.shape == (3, ld)
    assert qpos0.shape == state.qpos.shape and qvel0.shape == state.qvel.shape
    _capi.pg_env_reset(batch.handle, task.handle, state.c(), _ptr(task_state), _ptr(qpos0.contiguous()),
                       _ptr(qvel0.contiguous()), _ptr(cmd.contiguous()), _ptr(obs), _stream_ptr(stream))


def env_step(batch: Batch, task: Task, state: State, task_state: torch.Tensor, actions: torch.Tensor,
             cmd: torch.Tensor, qpos0: torch.Tensor, qvel0: torch.Tensor, n_substeps: int, obs: torch.Tensor,
             reward: torch.Tensor, done: torch.Tensor, truncated: torch.Tensor, terms: Optional[torch.Tensor] = None,
             stream=None, params: Optional[torch.Tensor] = None) -> None:
    """pg_env_step: targets, physics, reward, termination, reset and observation in one launch;
    params ([nrand][ld], optional): per-environment physical parameters as for step_dr."""
    ld = state.ld
    assert actions.dtype == torch.float32 and actions.is_contiguous() and actions.shape == (task.model.nu, ld)
    assert task_state.shape == (task.state_rows, ld) and obs.shape == (task.nobs, ld) and cmd.shape == (3, ld)
    assert reward.numel() >= ld and done.numel() >= ld and truncated.numel() >= ld
    assert terms is None or terms.shape == (task.nterms, ld)
    assert params is None or (params.dtype == torch.float32 and params.shape == (task.model.sizes.nrand, ld))
    _capi.pg_env_step(batch.handle, task.handle, state.c(), _ptr(task_state), _ptr(actions), _ptr(cmd.contiguous()),
                      _ptr(qpos0.contiguous()), _ptr(qvel0.contiguous()), int(n_substeps), _ptr(obs), _ptr(reward),
                      _ptr(done), _ptr(truncated), _ptr(terms), _ptr(params), _stream_ptr(stream))


def render(batch: Batch, state: State, scene: W.Scene, pixels: torch.Tensor, hits: Optional[torch.Tensor] = None,
           stream=None, cam_offset: Optional[torch.Tensor] = None, light_dir: Optional[torch.Tensor] = None,
           tint: Optional[torch.Tensor] = None) -> None:
    """pg_render: one ray-traced image per environment of the current state into pixels
    (uint8 [n][H][W][3] or float32 [n][H][W][3]); hits (int32 [n][H][W]) optional; per-environment
    camera offsets, light directions and colour tints ([3][ld] each) optional."""
    for t in (cam_offset, light_dir, tint):
        assert t is None or (t.dtype == torch.float32 and t.is_contiguous() and t.shape == (3, state.ld))
    fmt = _capi.PG_PIXELS_U8 if pixels.dtype == torch.uint8 else _capi.PG_PIXELS_F32
    assert pixels.dtype in (torch.uint8, torch.float32) and pixels.is_contiguous()
    assert pixels.shape == (state.n, scene.height, scene.width, 3)
    assert hits is None or (hits.dtype == torch.int32 and hits.shape == (state.n, scene.height, scene.width))
    rgb = np.ascontiguousarray(scene.geom_rgb, np.float32)
    f3 = lambda v: (C.c_float * 3)(*[float(x) for x in v])
    d = _capi.pg_render_desc(f3(scene.cam_pos), f3(scene.cam_lookat), f3(scene.cam_up), float(scene.fovy_deg),
                             int(scene.width), int(scene.height), f3(scene.light_dir), float(scene.ambient),
                             float(scene.diffuse), f3(scene.background), rgb.ctypes.data_as(C.c_void_p),
                             _ptr(cam_offset), _ptr(light_dir), _ptr(tint))
    _capi.pg_render(batch.handle, state.c(), d, fmt, _ptr(pixels), _ptr(hits), _stream_ptr(stream))


def reset(batch: Batch, state: State, qpos0: torch.Tensor, qvel0: torch.Tensor, mask: Optional[torch.Tensor] = None,
          stream=None) -> None:
    assert qpos0.shape == state.qpos.shape and qvel0.shape == state.qvel.shape
    _capi.pg_reset(batch.handle, state.c(), _ptr(mask), _ptr(qpos0.contiguous()), _ptr(qvel0.contiguous()),
                   _stream_ptr(stream))


def step(batch: Batch, state: State, ctrl: torch.Tensor, n_substeps: int, stream=None) -> None:
    assert ctrl.dtype == torch.float32 and ctrl.is_contiguous() and ctrl.shape[-1] == state.ld
    _capi.pg_step(batch.handle, state.c(), _ptr(ctrl), int(n_substeps), _stream_ptr(stream))


def step_ex(batch: Batch, state: State, ctrl: torch.Tensor, n_substeps: int,
            contact_force: Optional[torch.Tensor] = None, ncon: Optional[torch.Tensor] = None, stream=None) -> None:
    """pg_step_ex: the step with its optional outputs: contact_force [nslot, 3, ld] float32 (the last
    substep's force of every candidate contact slot in its contact frame), ncon [ld] int32."""
    assert ctrl.dtype == torch.float32 and ctrl.is_contiguous() and ctrl.shape[-1] == state.ld
    nslot = _capi.pg_batch_nslot(batch.handle)
    assert contact_force is None or (contact_force.dtype == torch.float32 and contact_force.is_contiguous() and
                                     tuple(contact_force.shape) == (nslot, 3, state.ld))
    assert ncon is None or (ncon.dtype == torch.int32 and ncon.numel() >= state.ld)
    out = _capi.pg_step_out(None if contact_force is None else contact_force.data_ptr(),
                            None if ncon is None else ncon.data_ptr())
    _capi.pg_step_ex(batch.handle, state.c(), _ptr(ctrl), int(n_substeps), out, _stream_ptr(stream))


def step_dr(batch: Batch, state: State, ctrl: torch.Tensor, params: torch.Tensor, n_substeps: int,
            stream=None) -> None:
    """pg_step_dr: the step with per-environment parameters params [nrand_max][ld] (friction
    scale, payload, centre-of-mass offsets, armature, calibration offsets, PD gain scales, link
    mass scales, friction-loss scales)."""
    assert ctrl.dtype == torch.float32 and ctrl.is_contiguous() and ctrl.shape[-1] == state.ld
    nrand = max(m.sizes.nrand for m in batch.models)
    assert params.dtype == torch.float32 and params.is_contiguous() and params.shape == (nrand, state.ld)
    _capi.pg_step_dr(batch.handle, state.c(), _ptr(ctrl), _ptr(params), int(n_substeps), _stream_ptr(stream))


def step_host(batch: Batch, state: State, ctrl_host: torch.Tensor, qpos_host: torch.Tensor, qvel_host: torch.Tensor,
              n_substeps: int, stream=None) -> None:
    _capi.pg_step_host(batch.handle, state.c(), _ptr(ctrl_host), _ptr(qpos_host), _ptr(qvel_host), int(n_substeps),
                       _stream_ptr(stream))


def rollout_host(batch: Batch, state: State, ctrl_host: torch.Tensor, qpos_host: torch.Tensor, qvel_host: torch.Tensor,
                 n_substeps: int, stream=None) -> None:
    """pg_rollout_host: T = ctrl_host.shape[0] control steps from host buffers (pinned, CPU tensors
    [T][nu_max][ld], [T][nq_max][ld], [T][nv_max][ld]), transfers overlapped with the steps."""
    T = ctrl_host.shape[0]
    for t, rows in ((ctrl_host, max(batch.nu_max, 1)), (qpos_host, batch.nq_max), (qvel_host, batch.nv_max)):
        assert t.device.type == "cpu" and t.dtype == torch.float32 and t.is_contiguous()
        assert t.shape[0] == T and t.shape[-1] == state.ld and t.shape[1] >= (rows if t is not ctrl_host else batch.nu_max)
    _capi.pg_rollout_host(batch.handle, state.c(), _ptr(ctrl_host), _ptr(qpos_host), _ptr(qvel_host), int(T),
                          int(n_substeps), _stream_ptr(stream))


def step_vjp(batch: Batch, ckpt: State, ctrl: torch.Tensor, n_substeps: int, g_qpos: Optional[torch.Tensor],
             g_qvel: Optional[torch.Tensor], adj_qpos: torch.Tensor, adj_qvel: torch.Tensor, g_ctrl: torch.Tensor,
             g_param: torch.Tensor, stream=None) -> None:
    """pg_step_vjp over the K = ctrl.shape[0] control steps that start from `ckpt` (see include/pg.h):
    adj_qpos / adj_qvel in: adjoint after the last step, out: adjoint of ckpt; g_ctrl [K, nu_max, ld]
    written; g_param [nparam_max, ld] accumulated."""
    K = ctrl.shape[0]
    for t, shape in ((ctrl, (K, max(batch.nu_max, 1), ckpt.ld)), (adj_qpos, (batch.nq_max, ckpt.ld)),
                     (adj_qvel, (batch.nv_max, ckpt.ld)), (g_ctrl, (K, max(batch.nu_max, 1), ckpt.ld)),
                     (g_param, (batch.nparam_max, ckpt.ld))):
        assert t.dtype == torch.float32 and t.is_contiguous() and tuple(t.shape) == shape, (t.shape, shape)
    for t, rows in ((g_qpos, batch.nq_max), (g_qvel, batch.nv_max)):
        assert t is None or (t.dtype == torch.float32 and t.is_contiguous() and tuple(t.shape) == (K, rows, ckpt.ld))
    _capi.pg_step_vjp(batch.handle, ckpt.c(), _ptr(ctrl), K, int(n_substeps), _ptr(g_qpos), _ptr(g_qvel),
                      _ptr(adj_qpos), _ptr(adj_qvel), _ptr(g_ctrl), _ptr(g_param), _stream_ptr(stream))


DEBUG_FIELDS = ["xpos", "xmat", "xcom", "M", "bias", "passive", "actuator", "a0", "contacts", "nrow", "rows", "qacc",
                "iterations", "status", "qpos_next", "qvel_next"]


def debug_layout(sizes) -> List[int]:
    nb, nv, nq, ns, nr = sizes.nbody, sizes.nv, sizes.nq, sizes.nslot, sizes.nrow_max
    lens = [3 * nb, 9 * nb, 3 * nb, nv * nv, nv, nv, nv, nv, 14 * ns, 1, nr * (nv + 7), nv, 1, 1, nq, nv]
    return list(np.cumsum([0] + lens))


def debug_substep(batch: Batch, state: State, ctrl: torch.Tensor, env: int, stream=None) -> dict:
    """Run one substep of env `env` and return its intermediates (numpy)."""
    k = max(i for i in range(len(batch.models)) if batch.env_off[i] <= env)
    sz = batch.models[k].sizes
    off = debug_layout(sz)
    out = torch.zeros(off[-1], dtype=torch.float32, device=state.qpos.device)
    _capi.pg_debug_substep(batch.handle, state.c(), _ptr(ctrl), int(env), _ptr(out), _stream_ptr(stream))
    torch.cuda.synchronize()
    o = out.cpu().numpy().astype(np.float64)
    r = {name: o[off[i]:off[i + 1]] for i, name in enumerate(DEBUG_FIELDS)}
    nv, nb = sz.nv, sz.nbody
    r["xpos"] = r["xpos"].reshape(nb, 3)
    r["xmat"] = r["xmat"].reshape(nb, 3, 3)
    r["xcom"] = r["xcom"].reshape(nb, 3)
    r["M"] = r["M"].reshape(nv, nv)
    r["contacts"] = r["contacts"].reshape(sz.nslot, 14)
    r["nrow"] = int(r["nrow"][0])
    r["rows"] = r["rows"].reshape(sz.nrow_max, nv + 7)[: r["nrow"]]
    r["iterations"] = int(r["iterations"][0])
    r["status"] = int(r["status"][0])
    return r


def to_soa(x: np.ndarray, ld: int, rows: Optional[int] = None) -> np.ndarray:
    """[N, k] env-major -> [rows, ld] coordinate-major (zero padded)."""
    n, k = x.shape
    out = np.zeros((rows if rows is not None else k, ld), np.float32)
    out[:k, :n] = x.T
    return out
