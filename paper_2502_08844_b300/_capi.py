"""ctypes binding of the C ABI in include/pg.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  The shared library is the
in-tree `libpg.so`; importing this module fails loudly when it is missing (there is no
fallback implementation of the step).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpg.so")

PG_OK, PG_EINVAL, PG_ENOMEM, PG_ECUDA, PG_EUNSUPPORTED, PG_ECAPACITY = 0, -1, -2, -3, -4, -5
PG_STATUS_NAN, PG_STATUS_NOT_CONVERGED, PG_STATUS_CAPACITY, PG_STATUS_WARM_RESET = 1, 2, 4, 8

_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int)


class pg_model_desc(C.Structure):
    _fields_ = [
        ("nbody", C.c_int), ("njnt", C.c_int), ("ngeom", C.c_int), ("npair", C.c_int), ("nu", C.c_int),
        ("body_parent", _ip), ("body_pos", _fp), ("body_quat", _fp), ("body_mass", _fp),
        ("body_ipos", _fp), ("body_inertia", _fp), ("body_geom_inertia", _ip),
        ("jnt_type", _ip), ("jnt_body", _ip), ("jnt_pos", _fp), ("jnt_axis", _fp),
        ("jnt_limited", _ip), ("jnt_range", _fp),
        ("dof_damping", _fp), ("dof_armature", _fp), ("dof_rotor", _fp),
        ("geom_type", _ip), ("geom_body", _ip), ("geom_pos", _fp), ("geom_quat", _fp),
        ("geom_size", _fp), ("geom_mass", _fp),
        ("pair_geom", _ip), ("pair_friction", _fp), ("pair_condim", _ip),
        ("act_type", _ip), ("act_jnt", _ip), ("act_gear", _fp), ("act_kp", _fp), ("act_kd", _fp),
        ("act_ctrllimited", _ip), ("act_ctrlrange", _fp),
        ("timestep", C.c_float), ("gravity", _fp), ("iterations", C.c_int), ("cone", C.c_int),
        ("impratio", C.c_float), ("solref", _fp), ("solimp", _fp), ("margin", C.c_float),
        ("max_contacts", C.c_int), ("substeps", C.c_int),
        ("hfield_nrow", C.c_int), ("hfield_ncol", C.c_int), ("hfield_data", _fp),
        ("act_forcelimited", _ip), ("act_forcerange", _fp), ("dof_frictionloss", _fp),
        ("nmesh", C.c_int), ("mesh_vertadr", _ip), ("mesh_vertnum", _ip), ("mesh_vert", _fp),
        ("mesh_faceadr", _ip), ("mesh_facenum", _ip), ("mesh_face", _ip), ("geom_meshid", _ip),
    ]


class pg_model_sizes(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("nq", "nv", "nu", "nbody", "njnt", "ngeom", "npair", "nslot", "nrow_max",
                                        "max_contacts", "workspace_bytes", "debug_floats",
                                        "adjoint_workspace_bytes", "nparam", "nrand")]


class pg_state(C.Structure):
    _fields_ = [("qpos", C.c_void_p), ("qvel", C.c_void_p), ("qacc_warm", C.c_void_p), ("status", C.c_void_p),
                ("n", C.c_int64), ("ld", C.c_int64), ("stats", C.c_void_p)]


PG_NTERMS = 15
PG_MAX_FEET = 8


class pg_task_desc(C.Structure):
    _fields_ = [("action_mode", C.c_int), ("action_scale", C.c_float), ("q_default", C.c_void_p),
                ("nfeet", C.c_int), ("foot_geom", C.c_void_p), ("contact_height", C.c_float),
                ("clearance_height", C.c_float), ("sigma_lin_vel", C.c_float), ("sigma_ang_vel", C.c_float),
                ("air_time_min", C.c_float), ("air_time_max", C.c_float), ("weight", C.c_float * PG_NTERMS),
                ("episode_length", C.c_int)]


class pg_task_sizes(C.Structure):
    _fields_ = [("nobs", C.c_int), ("nterms", C.c_int), ("state_rows", C.c_int)]


PG_PIXELS_U8, PG_PIXELS_F32 = 0, 1

PG_SPEC_BRANCH = 1
PG_SPEC_BRANCH_WARP = 2
PG_PRECOMPILE_WIDTH_ONLY = 4
PG_KERNEL_GENERIC, PG_KERNEL_SPECIALISED, PG_KERNEL_SPECIALISED_PARTS, PG_KERNEL_BRANCH = 0, 1, 2, 3
KERNEL_NAMES = {0: "generic", 1: "specialised", 2: "specialised per model", 3: "branch-parallel"}


class pg_step_out(C.Structure):
    _fields_ = [("contact_force", C.c_void_p), ("ncon", C.c_void_p)]


class pg_kernel_info(C.Structure):
    _fields_ = [("kernel", C.c_int), ("lanes_per_env", C.c_int), ("branches", C.c_int), ("reason", C.c_char * 160),
                ("branch_parts", C.c_int), ("sync", C.c_int), ("branch_dr", C.c_int), ("branch_tape", C.c_int),
                ("envs_per_warp", C.c_int)]


class pg_render_desc(C.Structure):
    _fields_ = [("cam_pos", C.c_float * 3), ("cam_lookat", C.c_float * 3), ("cam_up", C.c_float * 3),
                ("fovy_deg", C.c_float), ("width", C.c_int), ("height", C.c_int), ("light_dir", C.c_float * 3),
                ("ambient", C.c_float), ("diffuse", C.c_float), ("background", C.c_float * 3),
                ("geom_rgb", C.c_void_p), ("env_cam_offset", C.c_void_p), ("env_light_dir", C.c_void_p),
                ("env_tint", C.c_void_p)]


EXPORTS = ["pg_model_compile", "pg_model_info", "pg_model_free", "pg_batch_compile", "pg_batch_info",
           "pg_batch_free", "pg_reset", "pg_step", "pg_step_dr", "pg_debug_substep", "pg_step_host", "pg_rollout_host", "pg_step_vjp",
           "pg_step_vjp_noalloc", "pg_batch_specialize", "pg_batch_specialize_ex", "pg_batch_kernel",
           "pg_step_ex", "pg_batch_nslot", "pg_batch_reserve_vjp",
           "pg_model_branch_plan", "pg_model_precompile", "pg_task_compile", "pg_task_info", "pg_task_free",
           "pg_env_reset", "pg_env_step", "pg_render", "pg_last_error"]

if not os.path.exists(LIB_PATH):
    raise ImportError("libpg.so is not built (run `python -m paper_2502_08844_b300.build` or "
                      "__graft_entry__.build()); there is no fallback implementation of the step")

_lib = C.CDLL(LIB_PATH)

_lib.pg_last_error.restype = C.c_char_p
_lib.pg_last_error.argtypes = []
_lib.pg_model_compile.argtypes = [C.POINTER(pg_model_desc), C.POINTER(C.c_void_p)]
_lib.pg_model_info.argtypes = [C.c_void_p, C.POINTER(pg_model_sizes)]
_lib.pg_model_free.argtypes = [C.c_void_p]
_lib.pg_model_free.restype = None
_lib.pg_batch_compile.argtypes = [C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.c_int, C.c_int, C.POINTER(C.c_void_p)]
_lib.pg_batch_info.argtypes = [C.c_void_p, C.POINTER(C.c_int64), _ip, _ip, _ip]
_lib.pg_batch_free.argtypes = [C.c_void_p]
_lib.pg_batch_free.restype = None
_lib.pg_reset.argtypes = [C.c_void_p, C.POINTER(pg_state), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
_lib.pg_step.argtypes = [C.c_void_p, C.POINTER(pg_state), C.c_void_p, C.c_int, C.c_void_p]
_lib.pg_step_dr.argtypes = [C.c_void_p, C.POINTER(pg_state), C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
_lib.pg_debug_substep.argtypes = [C.c_void_p, C.POINTER(pg_state), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
_lib.pg_step_host.argtypes = [C.c_void_p, C.POINTER(pg_state), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
_lib.pg_rollout_host.argtypes = [C.c_void_p, C.POINTER(pg_state), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                 C.c_void_p]
_lib.pg_step_vjp.argtypes = [C.c_void_p, C.POINTER(pg_state), C.c_void_p, C.c_int, C.c_int] + [C.c_void_p] * 7
_lib.pg_batch_specialize.argtypes = [C.c_void_p]
_lib.pg_batch_specialize_ex.argtypes = [C.c_void_p, C.c_uint]
_lib.pg_step_ex.argtypes = [C.c_void_p, C.POINTER(pg_state), C.c_void_p, C.c_int, C.POINTER(pg_step_out), C.c_void_p]
_lib.pg_batch_nslot.argtypes = [C.c_void_p]
_lib.pg_batch_reserve_vjp.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64]
_lib.pg_batch_kernel.argtypes = [C.c_void_p, C.POINTER(pg_kernel_info)]
_lib.pg_model_branch_plan.argtypes = [C.c_void_p, C.POINTER(pg_kernel_info)]
_lib.pg_model_precompile.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_uint, C.c_char_p, _ip]
_lib.pg_step_vjp_noalloc.argtypes = [C.c_void_p, C.POINTER(pg_state), C.c_void_p, C.c_int, C.c_int] + [C.c_void_p] * 7
_lib.pg_task_compile.argtypes = [C.c_void_p, C.POINTER(pg_task_desc), C.POINTER(C.c_void_p)]
_lib.pg_task_info.argtypes = [C.c_void_p, C.POINTER(pg_task_sizes)]
_lib.pg_task_free.argtypes = [C.c_void_p]
_lib.pg_task_free.restype = None
_lib.pg_env_reset.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(pg_state)] + [C.c_void_p] * 6
_lib.pg_env_step.argtypes = ([C.c_void_p, C.c_void_p, C.POINTER(pg_state)] + [C.c_void_p] * 5 + [C.c_int] +
                             [C.c_void_p] * 7)
_lib.pg_render.argtypes = [C.c_void_p, C.POINTER(pg_state), C.POINTER(pg_render_desc), C.c_int, C.c_void_p,
                           C.c_void_p, C.c_void_p]
for _n in EXPORTS:
    if _n not in ("pg_last_error", "pg_model_free", "pg_batch_free"):
        getattr(_lib, _n).restype = C.c_int


class PgError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s failed (%d): %s" % (where, code, pg_last_error()))


def _check(rc: int, where: str) -> None:
    if rc != PG_OK:
        raise PgError(rc, where)


def pg_last_error() -> str:
    s = _lib.pg_last_error()
    return s.decode() if s else ""


def pg_model_compile(desc: pg_model_desc) -> C.c_void_p:
    out = C.c_void_p()
    _check(_lib.pg_model_compile(C.byref(desc), C.byref(out)), "pg_model_compile")
    return out


def pg_model_info(model) -> pg_model_sizes:
    s = pg_model_sizes()
    _check(_lib.pg_model_info(model, C.byref(s)), "pg_model_info")
    return s


def pg_model_free(model) -> None:
    _lib.pg_model_free(model)


def pg_batch_compile(models, counts, envs_per_cta: int = 0) -> C.c_void_p:
    arr = (C.c_void_p * len(models))(*[m.value for m in models])
    cnt = (C.c_int64 * len(counts))(*counts)
    out = C.c_void_p()
    _check(_lib.pg_batch_compile(arr, cnt, len(models), int(envs_per_cta), C.byref(out)), "pg_batch_compile")
    return out


def pg_batch_info(batch):
    n = C.c_int64(); nq = C.c_int(); nv = C.c_int(); nu = C.c_int()
    _check(_lib.pg_batch_info(batch, C.byref(n), C.byref(nq), C.byref(nv), C.byref(nu)), "pg_batch_info")
    return n.value, nq.value, nv.value, nu.value


def pg_batch_free(batch) -> None:
    _lib.pg_batch_free(batch)


def pg_reset(batch, state: pg_state, env_mask_ptr, qpos0_ptr, qvel0_ptr, stream) -> None:
    _check(_lib.pg_reset(batch, C.byref(state), env_mask_ptr, qpos0_ptr, qvel0_ptr, stream), "pg_reset")


def pg_step(batch, state: pg_state, ctrl_ptr, n_substeps: int, stream) -> None:
    _check(_lib.pg_step(batch, C.byref(state), ctrl_ptr, int(n_substeps), stream), "pg_step")


def pg_step_dr(batch, state: pg_state, ctrl_ptr, params_ptr, n_substeps: int, stream) -> None:
    _check(_lib.pg_step_dr(batch, C.byref(state), ctrl_ptr, params_ptr, int(n_substeps), stream), "pg_step_dr")


def pg_debug_substep(batch, state: pg_state, ctrl_ptr, env: int, out_ptr, stream) -> None:
    _check(_lib.pg_debug_substep(batch, C.byref(state), ctrl_ptr, int(env), out_ptr, stream), "pg_debug_substep")


def pg_rollout_host(batch, state: pg_state, ctrl_host_ptr, qpos_host_ptr, qvel_host_ptr, n_steps: int, n_substeps: int,
                    stream) -> None:
    _check(_lib.pg_rollout_host(batch, C.byref(state), ctrl_host_ptr, qpos_host_ptr, qvel_host_ptr, int(n_steps),
                                int(n_substeps), stream), "pg_rollout_host")


def pg_step_host(batch, state: pg_state, ctrl_host_ptr, qpos_host_ptr, qvel_host_ptr, n_substeps: int, stream) -> None:
    _check(_lib.pg_step_host(batch, C.byref(state), ctrl_host_ptr, qpos_host_ptr, qvel_host_ptr, int(n_substeps), stream),
           "pg_step_host")


def pg_step_vjp(batch, ckpt: pg_state, ctrl_ptr, n_steps: int, n_substeps: int, g_qpos_ptr, g_qvel_ptr, adj_qpos_ptr,
                adj_qvel_ptr, g_ctrl_ptr, g_param_ptr, stream) -> None:
    _check(_lib.pg_step_vjp(batch, C.byref(ckpt), ctrl_ptr, int(n_steps), int(n_substeps), g_qpos_ptr, g_qvel_ptr,
                            adj_qpos_ptr, adj_qvel_ptr, g_ctrl_ptr, g_param_ptr, stream), "pg_step_vjp")


def pg_step_vjp_noalloc(batch, ckpt: pg_state, ctrl_ptr, n_steps: int, n_substeps: int, g_qpos_ptr, g_qvel_ptr,
                        adj_qpos_ptr, adj_qvel_ptr, g_ctrl_ptr, g_param_ptr, stream) -> None:
    _check(_lib.pg_step_vjp_noalloc(batch, C.byref(ckpt), ctrl_ptr, int(n_steps), int(n_substeps), g_qpos_ptr,
                                    g_qvel_ptr, adj_qpos_ptr, adj_qvel_ptr, g_ctrl_ptr, g_param_ptr, stream),
           "pg_step_vjp_noalloc")


def pg_batch_specialize(batch) -> None:
    _check(_lib.pg_batch_specialize(batch), "pg_batch_specialize")


def pg_step_ex(batch, state: pg_state, ctrl_ptr, n_substeps: int, out, stream) -> None:
    _check(_lib.pg_step_ex(batch, C.byref(state), ctrl_ptr, n_substeps, None if out is None else C.byref(out), stream),
           "pg_step_ex")


def pg_batch_reserve_vjp(batch, n_steps: int, n_substeps: int, ld: int) -> None:
    _check(_lib.pg_batch_reserve_vjp(batch, n_steps, n_substeps, ld), "pg_batch_reserve_vjp")


def pg_batch_nslot(batch) -> int:
    return _lib.pg_batch_nslot(batch)


def pg_batch_specialize_ex(batch, flags: int) -> None:
    _check(_lib.pg_batch_specialize_ex(batch, flags), "pg_batch_specialize_ex")


def pg_batch_kernel(batch) -> pg_kernel_info:
    out = pg_kernel_info()
    _check(_lib.pg_batch_kernel(batch, C.byref(out)), "pg_batch_kernel")
    return out


def pg_model_branch_plan(model) -> pg_kernel_info:
    out = pg_kernel_info()
    _check(_lib.pg_model_branch_plan(model, C.byref(out)), "pg_model_branch_plan")
    return out


def pg_model_precompile(model, count: int, envs_per_cta: int, sms: int, flags: int, dir_) -> int:
    """dir_: a directory or None (the disk cache).  Returns the thread-per-environment kernels'
    width (environments per warp)."""
    w = C.c_int(0)
    _check(_lib.pg_model_precompile(model, int(count), int(envs_per_cta), int(sms), flags,
                                    None if dir_ is None else dir_.encode(), C.byref(w)), "pg_model_precompile")
    return w.value


def pg_task_compile(model, desc: pg_task_desc) -> C.c_void_p:
    out = C.c_void_p()
    _check(_lib.pg_task_compile(model, C.byref(desc), C.byref(out)), "pg_task_compile")
    return out


def pg_task_info(task) -> pg_task_sizes:
    s = pg_task_sizes()
    _check(_lib.pg_task_info(task, C.byref(s)), "pg_task_info")
    return s


def pg_task_free(task) -> None:
    _lib.pg_task_free(task)


def pg_env_reset(batch, task, state: pg_state, task_state_ptr, qpos0_ptr, qvel0_ptr, cmd_ptr, obs_ptr, stream) -> None:
    _check(_lib.pg_env_reset(batch, task, C.byref(state), task_state_ptr, qpos0_ptr, qvel0_ptr, cmd_ptr, obs_ptr,
                             stream), "pg_env_reset")


def pg_env_step(batch, task, state: pg_state, task_state_ptr, action_ptr, cmd_ptr, qpos0_ptr, qvel0_ptr,
                n_substeps: int, obs_ptr, reward_ptr, done_ptr, truncated_ptr, terms_ptr, params_ptr, stream) -> None:
    _check(_lib.pg_env_step(batch, task, C.byref(state), task_state_ptr, action_ptr, cmd_ptr, qpos0_ptr, qvel0_ptr,
                            int(n_substeps), obs_ptr, reward_ptr, done_ptr, truncated_ptr, terms_ptr, params_ptr,
                            stream), "pg_env_step")


def pg_render(batch, state: pg_state, desc: pg_render_desc, fmt: int, pixels_ptr, hits_ptr, stream) -> None:
    _check(_lib.pg_render(batch, C.byref(state), C.byref(desc), int(fmt), pixels_ptr, hits_ptr, stream), "pg_render")
