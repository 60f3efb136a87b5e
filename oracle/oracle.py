"""Python handle on the FP64 oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg import this
module.  It loads `liborc.so` (built from the C++ sources beside it) with ctypes and feeds it
the same float32-rounded model arrays and inputs the CUDA library receives, widened to
double.  Arrays here are environment-major ([env][coord]).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class _Desc(C.Structure):
    _fields_ = [
        ("nbody", C.c_int), ("njnt", C.c_int), ("ngeom", C.c_int), ("npair", C.c_int), ("nu", C.c_int),
        ("body_parent", _ip), ("body_pos", _dp), ("body_quat", _dp), ("body_mass", _dp),
        ("body_ipos", _dp), ("body_inertia", _dp), ("body_geom_inertia", _ip),
        ("jnt_type", _ip), ("jnt_body", _ip), ("jnt_pos", _dp), ("jnt_axis", _dp),
        ("jnt_limited", _ip), ("jnt_range", _dp),
        ("dof_damping", _dp), ("dof_armature", _dp), ("dof_rotor", _dp),
        ("geom_type", _ip), ("geom_body", _ip), ("geom_pos", _dp), ("geom_quat", _dp),
        ("geom_size", _dp), ("geom_mass", _dp),
        ("pair_geom", _ip), ("pair_friction", _dp), ("pair_condim", _ip),
        ("act_type", _ip), ("act_jnt", _ip), ("act_gear", _dp), ("act_kp", _dp), ("act_kd", _dp),
        ("act_ctrllimited", _ip), ("act_ctrlrange", _dp),
        ("timestep", C.c_double), ("gravity", _dp), ("iterations", C.c_int), ("cone", C.c_int),
        ("impratio", C.c_double), ("solref", _dp), ("solimp", _dp), ("margin", C.c_double),
        ("max_contacts", C.c_int),
        ("hfield_nrow", C.c_int), ("hfield_ncol", C.c_int), ("hfield_data", _dp),
        ("act_forcelimited", _ip), ("act_forcerange", _dp),
        ("dof_frictionloss", _dp),
        ("nmesh", C.c_int), ("mesh_vertadr", _ip), ("mesh_vertnum", _ip), ("mesh_vert", _dp),
        ("mesh_faceadr", _ip), ("mesh_facenum", _ip), ("mesh_face", _ip), ("geom_meshid", _ip),
    ]


_libs = {}


def lib(native: bool = False):
    """The oracle's library: the portable build, or (native=True) the -O3 -march=native build
    that the timed CPU legs use, compiled on the host that runs them."""
    if native not in _libs:
        path = _build.build(native=native)
        L = C.CDLL(path)
        L.orc_model_new.restype = C.c_void_p
        L.orc_model_new.argtypes = [C.POINTER(_Desc), C.c_char_p, C.c_int]
        L.orc_model_free.argtypes = [C.c_void_p]
        for name in ["orc_model_sizes", "orc_forward_layout"]:
            getattr(L, name).argtypes = [C.c_void_p, _ip]
        L.orc_model_massprops.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.orc_rollout.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _dp,
                                  C.POINTER(C.c_uint32), C.c_int, C.c_int, _dp, _dp]
        L.orc_forward.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, C.c_int, _dp]
        L.orc_inverse_dynamics.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.orc_mass_matrix.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_mass_matrix_crba.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_body_frames.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_geom_frames.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_energy.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.orc_momentum.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.orc_point_jacobian.argtypes = [C.c_void_p, _dp, C.c_int, _dp, _dp, _dp]
        L.orc_integrate_pos.argtypes = [C.c_void_p, _dp, _dp, C.c_double]
        L.orc_collide.argtypes = [C.c_int, _dp, _dp, _dp, C.c_int, _dp, _dp, _dp, _dp]
        L.orc_collide_hfield.argtypes = [_dp, _dp, _dp, C.c_int, C.c_int, _dp, C.c_int, _dp, _dp, _dp, _dp]
        L.orc_collide_mesh.argtypes = [C.c_int, _dp, _dp, _dp, C.c_int, C.c_int, _dp, C.c_int, _dp, C.c_int, _ip,
                                       _dp, _dp, _dp]
        L.orc_solve.argtypes = [C.c_int, _dp, _dp, C.c_int, _dp, _dp, _dp, _dp, C.c_int, _dp, _dp, _ip, _ip, _dp]
        L.orc_cost.restype = C.c_double
        L.orc_cost.argtypes = [C.c_int, _dp, _dp, C.c_int, _dp, _dp, _dp, _dp, _ip, _dp]
        L.orc_cone_cost.restype = C.c_double
        L.orc_cone_cost.argtypes = [_dp, C.c_double, C.c_double, _dp, _dp, _ip]
        L.orc_impedance.restype = C.c_double
        L.orc_impedance.argtypes = [C.c_double, _dp]
        L.orc_solid_inertia.argtypes = [C.c_int, _dp, C.c_double, _dp]
        L.orc_rotor_armature.restype = C.c_double
        L.orc_rotor_armature.argtypes = [C.c_double, C.c_double, C.c_double]
        _libs[native] = L
    return _libs[native]


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _pd(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _pi(a: np.ndarray):
    return a.ctypes.data_as(_ip)


class OracleModel:
    """A compiled oracle model built from a workloads.Model (float32 values widened to double)."""

    LAYOUT = ["xpos", "xmat", "xcom", "M", "bias", "passive", "actuator", "a0", "contacts", "nrow", "rows",
              "qacc", "iterations", "status", "qpos_next", "qvel_next"]

    def __init__(self, m, native: bool = False):
        """native: use the -O3 -march=native build (the timed CPU legs); results are the same
        method in FP64, rounding aside."""
        L = lib(native)
        self.L = L
        self.src = m
        keep = {}

        def D(name, arr):
            keep[name] = _d(arr)
            return _pd(keep[name])

        def I(name, arr):
            keep[name] = _i(arr)
            return _pi(keep[name])

        desc = _Desc(
            m.nbody, m.njnt, m.ngeom, m.npair, m.nu,
            I("bp", m.body_parent), D("bpos", m.body_pos), D("bq", m.body_quat), D("bm", m.body_mass),
            D("bip", m.body_ipos), D("bin", m.body_inertia), I("bgi", m.body_geom_inertia),
            I("jt", m.jnt_type), I("jb", m.jnt_body), D("jp", m.jnt_pos), D("ja", m.jnt_axis),
            I("jl", m.jnt_limited), D("jr", m.jnt_range),
            D("dd", m.dof_damping), D("da", m.dof_armature), D("dr", m.dof_rotor),
            I("gt", m.geom_type), I("gb", m.geom_body), D("gp", m.geom_pos), D("gq", m.geom_quat),
            D("gs", m.geom_size), D("gm", m.geom_mass),
            I("pg", m.pair_geom if m.npair else np.zeros((0, 2))), D("pf", m.pair_friction), I("pc", m.pair_condim),
            I("at", m.act_type), I("aj", m.act_jnt), D("ag", m.act_gear), D("akp", m.act_kp), D("akd", m.act_kd),
            I("acl", m.act_ctrllimited), D("acr", m.act_ctrlrange),
            float(m.timestep), D("grav", m.gravity), int(m.iterations), int(m.cone), float(m.impratio),
            D("sref", m.solref), D("simp", m.solimp), float(m.margin), int(m.max_contacts),
            0 if getattr(m, "hfield", None) is None else int(m.hfield.shape[0]),
            0 if getattr(m, "hfield", None) is None else int(m.hfield.shape[1]),
            None if getattr(m, "hfield", None) is None else D("hf", m.hfield),
            None if getattr(m, "act_forcelimited", None) is None else I("afl", m.act_forcelimited),
            None if getattr(m, "act_forcerange", None) is None else D("afr", m.act_forcerange),
            None if getattr(m, "dof_frictionloss", None) is None else D("dfl", m.dof_frictionloss),
            getattr(m, "nmesh", 0),
            *((I("mva", m.mesh_vertadr), I("mvn", m.mesh_vertnum), D("mv", m.mesh_vert), I("mfa", m.mesh_faceadr),
               I("mfn", m.mesh_facenum), I("mf", m.mesh_face), I("gmi", m.geom_meshid))
              if getattr(m, "nmesh", 0) else (None,) * 7),
        )
        err = C.create_string_buffer(256)
        h = L.orc_model_new(C.byref(desc), err, 256)
        if not h:
            raise ValueError("oracle model: " + err.value.decode())
        self.h = C.c_void_p(h)
        s = np.zeros(11, np.int32)
        L.orc_model_sizes(self.h, _pi(s))
        (self.nq, self.nv, self.nu, self.nbody, self.ngeom, self.nslot, self.nrow_max, self.njnt, self.npair,
         self.nlimited, self.max_contacts) = [int(x) for x in s]
        off = np.zeros(17, np.int32)
        L.orc_forward_layout(self.h, _pi(off))
        self.off = [int(x) for x in off]

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None and getattr(self, "L", None) is not None:
                self.L.orc_model_free(self.h)
        except Exception:
            pass

    # ---- model tables --------------------------------------------------------------
    def massprops(self):
        mass = np.zeros(self.nbody); ipos = np.zeros((self.nbody, 3)); inertia = np.zeros((self.nbody, 6))
        arm = np.zeros(self.nv)
        self.L.orc_model_massprops(self.h, _pd(mass), _pd(ipos), _pd(inertia), _pd(arm))
        return mass, ipos, inertia, arm

    # ---- stepping ------------------------------------------------------------------
    def rollout(self, qpos, qvel, ctrl, n_substeps: int, qacc_warm=None, solver_cap: Optional[int] = None,
                nthreads: int = 1, trajectory: bool = False):
        """Advance envs (qpos [N,nq], qvel [N,nv]) through ctrl [T,N,nu].  Returns
        (qpos, qvel, qacc_warm, status) and, with trajectory=True, per-step qpos/qvel [T,N,*]."""
        qpos = _d(qpos).copy(); qvel = _d(qvel).copy()
        N = qpos.shape[0]
        ctrl = _d(ctrl)
        T = ctrl.shape[0]
        assert ctrl.shape == (T, N, self.nu) or (self.nu == 0 and ctrl.size == 0)
        warm = np.zeros((N, self.nv)) if qacc_warm is None else _d(qacc_warm).copy()
        status = np.zeros(N, np.uint32)
        cap = self.src.iterations if solver_cap is None else solver_cap
        tq = np.zeros((T, N, self.nq)) if trajectory else None
        tv = np.zeros((T, N, self.nv)) if trajectory else None
        if ctrl.size == 0:
            ctrl = np.zeros((T, N, max(self.nu, 1)))
        r = self.L.orc_rollout(self.h, N, T, int(n_substeps), _pd(qpos), _pd(qvel), _pd(warm), _pd(ctrl),
                              status.ctypes.data_as(C.POINTER(C.c_uint32)), int(cap), int(nthreads),
                              _pd(tq) if trajectory else None, _pd(tv) if trajectory else None)
        if r != 0:
            raise ValueError("orc_rollout failed")
        if trajectory:
            return qpos, qvel, warm, status, tq, tv
        return qpos, qvel, warm, status

    def forward(self, qpos, qvel, qacc_warm=None, ctrl=None, solver_cap: Optional[int] = None) -> dict:
        """One substep of one env; returns every intermediate of the diagnostic record."""
        qpos = _d(qpos); qvel = _d(qvel)
        warm = np.zeros(self.nv) if qacc_warm is None else _d(qacc_warm)
        u = np.zeros(max(self.nu, 1)) if ctrl is None else _d(ctrl)
        out = np.zeros(self.off[16])
        cap = self.src.iterations if solver_cap is None else solver_cap
        self.L.orc_forward(self.h, _pd(qpos), _pd(qvel), _pd(warm), _pd(u), int(cap), _pd(out))
        return self.unpack(out)

    def unpack(self, out: np.ndarray) -> dict:
        o, nv = self.off, self.nv
        r = {k: out[o[i]:o[i + 1]].copy() for i, k in enumerate(self.LAYOUT)}
        r["xpos"] = r["xpos"].reshape(self.nbody, 3)
        r["xmat"] = r["xmat"].reshape(self.nbody, 3, 3)
        r["xcom"] = r["xcom"].reshape(self.nbody, 3)
        r["M"] = r["M"].reshape(nv, nv)
        r["contacts"] = r["contacts"].reshape(self.nslot, 14)
        r["nrow"] = int(r["nrow"][0])
        r["rows"] = r["rows"].reshape(self.nrow_max, nv + 7)[: r["nrow"]]
        r["iterations"] = int(r["iterations"][0])
        r["status"] = int(r["status"][0])
        return r

    # ---- pins ------------------------------------------------------------------------
    def inverse_dynamics(self, qpos, qvel, qacc):
        tau = np.zeros(self.nv)
        self.L.orc_inverse_dynamics(self.h, _pd(_d(qpos)), _pd(_d(qvel)), _pd(_d(qacc)), _pd(tau))
        return tau

    def mass_matrix(self, qpos):
        M = np.zeros((self.nv, self.nv))
        self.L.orc_mass_matrix(self.h, _pd(_d(qpos)), _pd(M))
        return M

    def mass_matrix_crba(self, qpos):
        """The mass matrix by CRBA (the method the flop count takes), against mass_matrix's
        kinetic-energy definition."""
        M = np.zeros((self.nv, self.nv))
        self.L.orc_mass_matrix_crba(self.h, _pd(_d(qpos)), _pd(M))
        return M

    def body_frames(self, qpos):
        out = np.zeros((self.nbody, 15))
        self.L.orc_body_frames(self.h, _pd(_d(qpos)), _pd(out))
        return out[:, :9].reshape(-1, 3, 3), out[:, 9:12], out[:, 12:15]

    def geom_frames(self, qpos):
        out = np.zeros((self.ngeom, 12))
        self.L.orc_geom_frames(self.h, _pd(_d(qpos)), _pd(out))
        return out[:, :9].reshape(-1, 3, 3), out[:, 9:12]

    def energy(self, qpos, qvel):
        out = np.zeros(2)
        self.L.orc_energy(self.h, _pd(_d(qpos)), _pd(_d(qvel)), _pd(out))
        return out[0], out[1]

    def momentum(self, qpos, qvel):
        out = np.zeros(9)
        self.L.orc_momentum(self.h, _pd(_d(qpos)), _pd(_d(qvel)), _pd(out))
        return out[:3], out[3:6], out[6:9]

    def point_jacobian(self, qpos, body, point):
        Jv = np.zeros((3, self.nv)); Jw = np.zeros((3, self.nv))
        self.L.orc_point_jacobian(self.h, _pd(_d(qpos)), int(body), _pd(_d(point)), _pd(Jv), _pd(Jw))
        return Jv, Jw

    def integrate_pos(self, qpos, qvel, dt):
        q = _d(qpos).copy()
        self.L.orc_integrate_pos(self.h, _pd(q), _pd(_d(qvel)), float(dt))
        return q


def collide(t1, R1, p1, s1, t2, R2, p2, s2):
    """Model-free primitive collision; returns [npts, 13] (dist, pos3, n3, t1 3, t2 3)."""
    out = np.zeros((4, 13))
    n = lib().orc_collide(int(t1), _pd(_d(R1)), _pd(_d(p1)), _pd(_d(list(s1) + [0] * (3 - len(s1)))), int(t2),
                          _pd(_d(R2)), _pd(_d(p2)), _pd(_d(list(s2) + [0] * (3 - len(s2)))), _pd(out))
    if n < 0:
        raise ValueError("unsupported pair")
    return out[:n]


def collide_hfield(R1, p1, size, elev, t2, R2, p2, s2):
    """Model-free heightfield (geom1) against a sphere or capsule; [npts, 13] records as collide()."""
    elev = _d(elev)
    out = np.zeros((4, 13))
    n = lib().orc_collide_hfield(_pd(_d(R1)), _pd(_d(p1)), _pd(_d(size)), int(elev.shape[0]), int(elev.shape[1]),
                                 _pd(np.ascontiguousarray(elev)), int(t2), _pd(_d(R2)), _pd(_d(p2)),
                                 _pd(_d(list(s2) + [0] * (3 - len(s2)))), _pd(out))
    if n < 0:
        raise ValueError("unsupported pair")
    return out[:n]


def collide_mesh(R1, p1, R2, p2, vert, face, size=None, elev=None):
    """Model-free plane (elev None) or heightfield (size, elev) as geom1 against a convex mesh
    (vertices [n, 3], outward triangles [f, 3]) as geom2; [4, 13] records as collide()."""
    vert = np.ascontiguousarray(_d(vert))
    face = np.ascontiguousarray(np.asarray(face, np.int32))
    out = np.zeros((4, 13))
    hf = elev is not None
    e = np.ascontiguousarray(_d(elev)) if hf else None
    n = lib().orc_collide_mesh(4 if hf else 0, _pd(_d(R1)), _pd(_d(p1)), _pd(_d(size)) if hf else None,
                               int(e.shape[0]) if hf else 0, int(e.shape[1]) if hf else 0, _pd(e) if hf else None,
                               int(vert.shape[0]), _pd(vert), int(face.shape[0]), _pi(face), _pd(_d(R2)), _pd(_d(p2)),
                               _pd(out))
    if n < 0:
        raise ValueError("unsupported pair or mesh")
    return out


def _kinds(kind, mu, nr):
    if kind is None:
        return None, None, None
    k = np.ascontiguousarray(np.asarray(kind, np.int32)).reshape(nr)
    m = _d(mu).reshape(nr)
    return k, k.ctypes.data_as(_ip), _pd(m)


def solve(M, a0, J, aref, D, warm=None, cap=-1, kind=None, mu=None):
    """Newton solve on raw data; cap < 0 runs to convergence.  Returns (qacc, force, iters, converged).
    kind / mu (optional, per row): 0 scalar one-sided row, 1 elliptic normal row followed by its
    two tangent rows (kind 2), with the contact's friction in mu; 3 friction-loss row with its
    force bound in mu."""
    M = _d(M); a0 = _d(a0); J = _d(J).reshape(-1, M.shape[0]); aref = _d(aref); D = _d(D)
    nv, nr = M.shape[0], J.shape[0]
    qacc = np.zeros(nv); force = np.zeros(max(nr, 1)); it = C.c_int(0)
    keep, kp, mp = _kinds(kind, mu, nr)
    conv = lib().orc_solve(nv, _pd(M), _pd(a0), nr, _pd(J), _pd(aref), _pd(D),
                           _pd(_d(warm)) if warm is not None else None, int(cap), _pd(qacc), _pd(force), C.byref(it),
                           kp, mp)
    return qacc, force[:nr], it.value, bool(conv)


def cost(M, a0, J, aref, D, a, kind=None, mu=None):
    M = _d(M); J = _d(J).reshape(-1, M.shape[0])
    keep, kp, mp = _kinds(kind, mu, J.shape[0])
    return lib().orc_cost(M.shape[0], _pd(M), _pd(_d(a0)), J.shape[0], _pd(J), _pd(_d(aref)), _pd(_d(D)), _pd(_d(a)),
                          kp, mp)


def cone_cost(x, D, mu):
    """Elliptic contact cost s(x) with its gradient, Hessian and zone (0 free, 1 boundary, 2 full)."""
    g = np.zeros(3); H = np.zeros(9); z = C.c_int(0)
    f = lib().orc_cone_cost(_pd(_d(x)), float(D), float(mu), _pd(g), _pd(H), C.byref(z))
    return f, g, H.reshape(3, 3), z.value


def impedance(r, solimp):
    return lib().orc_impedance(float(r), _pd(_d(solimp)))


def solid_inertia(gtype, size, mass):
    out = np.zeros(3)
    lib().orc_solid_inertia(int(gtype), _pd(_d(list(size) + [0] * (3 - len(size)))), float(mass), _pd(out))
    return out


def rotor_armature(kg, mr, rr):
    return lib().orc_rotor_armature(float(kg), float(mr), float(rr))


def _setup_grad_api(L=None):
    L = lib() if L is None else L
    if getattr(L, "_grad_ready", False):
        return L
    L.orc_rollout_loss.restype = C.c_double
    L.orc_rollout_loss.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_rollout_grad.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp,
                                   _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_step_vjp.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L._grad_ready = True
    return L


def tracking_loss_weights(om: "OracleModel", z_target=0.27, v_target=(0.5, 0.0, 0.0)):
    """Weights/targets of the torso-tracking loss sum_t (z_t - z*)^2 + |v_t - v*|^2 (free-joint
    height qpos[2] and world linear velocity qvel[0:3])."""
    wq = np.zeros(om.nq); qs = np.zeros(om.nq); wv = np.zeros(om.nv); vs = np.zeros(om.nv)
    wq[2] = 1.0; qs[2] = z_target
    wv[:3] = 1.0; vs[:3] = v_target
    return wq, qs, wv, vs


def _opt(a):
    return None if a is None else _pd(_d(a))


def rollout_loss(om: "OracleModel", q0, v0, ctrl, n_substeps, weights, solver_cap=-1, mass=None, damping=None, kp=None):
    L = _setup_grad_api(om.L)
    ctrl = _d(ctrl).reshape(len(ctrl), om.nu)
    wq, qs, wv, vs = [_d(x) for x in weights]
    return L.orc_rollout_loss(om.h, _pd(_d(q0)), _pd(_d(v0)), _pd(ctrl), ctrl.shape[0], int(n_substeps), int(solver_cap),
                              _opt(mass), _opt(damping), _opt(kp), _pd(wq), _pd(qs), _pd(wv), _pd(vs))


def step_vjp(om: "OracleModel", q, v, u, n_substeps, bq, bv, solver_cap=-1, mass=None, damping=None, kp=None):
    """Reverse mode through one control step from (q, v) with controls u, given the adjoint (bq, bv)
    of the post-step state: dict with the pre-step adjoints q, v, the control adjoint u and the
    parameter adjoints mass, damping, kp (the warm start is a constant)."""
    L = _setup_grad_api(om.L)
    out = {"q": _d(bq).copy(), "v": _d(bv).copy(), "u": np.zeros(om.nu), "mass": np.zeros(om.nbody),
           "damping": np.zeros(om.nv), "kp": np.zeros(om.nu)}
    L.orc_step_vjp(om.h, _pd(_d(q)), _pd(_d(v)), _pd(_d(u).reshape(om.nu)), int(n_substeps), int(solver_cap),
                   _opt(mass), _opt(damping), _opt(kp), _pd(out["q"]), _pd(out["v"]), _pd(out["u"]), _pd(out["mass"]),
                   _pd(out["damping"]), _pd(out["kp"]))
    return out


def rollout_grad(om: "OracleModel", q0, v0, ctrl, n_substeps, weights, solver_cap=-1, mass=None, damping=None, kp=None):
    """Reverse-mode gradient of rollout_loss: dict with loss, q0, v0, u [T,nu], mass, damping, kp."""
    L = _setup_grad_api(om.L)
    ctrl = _d(ctrl).reshape(len(ctrl), om.nu)
    T = ctrl.shape[0]
    wq, qs, wv, vs = [_d(x) for x in weights]
    out = {"q0": np.zeros(om.nq), "v0": np.zeros(om.nv), "u": np.zeros((T, om.nu)), "mass": np.zeros(om.nbody),
           "damping": np.zeros(om.nv), "kp": np.zeros(om.nu)}
    loss = C.c_double(0)
    L.orc_rollout_grad(om.h, _pd(_d(q0)), _pd(_d(v0)), _pd(ctrl), T, int(n_substeps), int(solver_cap), _opt(mass),
                       _opt(damping), _opt(kp), _pd(wq), _pd(qs), _pd(wv), _pd(vs), _pd(out["q0"]), _pd(out["v0"]),
                       _pd(out["u"]), _pd(out["mass"]), _pd(out["damping"]), _pd(out["kp"]), C.byref(loss))
    out["loss"] = loss.value
    return out


COUNT_PHASES = ("kinematics", "mass_matrix", "bias", "smooth", "collision", "rows", "solve", "integrate", "force_output")
COUNT_KINDS = ("add", "mul", "div", "sqrt", "trans")


def count_selftest(which: int, n: int) -> float:
    """Counted flops of a textbook kernel on the counting scalar (see orc_count_selftest)."""
    L = lib()
    L.orc_count_selftest.argtypes = [C.c_int, C.c_int, _dp]
    out = np.zeros(1)
    if L.orc_count_selftest(int(which), int(n), _pd(out)) != 0:
        raise ValueError("orc_count_selftest failed")
    return float(out[0])


def count_substeps(om: "OracleModel", qpos, qvel, qacc_warm, ctrl, n_substeps: int, solver_cap: Optional[int] = None):
    """The oracle on its counting scalar (orc_count.hpp) over n_substeps substeps of one
    environment: (counts [S, phase, kind], rows [S], iters [S], final qpos, qvel, warm).  kind:
    add, mul, div, sqrt, transcendental; the factorisations counted are the leaves-first L^T D L."""
    L = om.L
    if not getattr(L, "_count_ready", False):
        L.orc_count_substeps.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, C.c_int, C.c_int, _dp,
                                         C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L._count_ready = True
    q, v, w = _d(qpos).copy(), _d(qvel).copy(), _d(qacc_warm).copy()
    u = _d(ctrl).reshape(-1).copy() if om.nu else np.zeros(1)
    S = int(n_substeps)
    counts = np.zeros((S, len(COUNT_PHASES), len(COUNT_KINDS)))
    rows = np.zeros(S, np.int32)
    iters = np.zeros(S, np.int32)
    cap = om.src.iterations if solver_cap is None else solver_cap
    r = L.orc_count_substeps(om.h, _pd(q), _pd(v), _pd(w), _pd(u), S, int(cap), _pd(counts), _pi(rows), _pi(iters))
    if r != 0:
        raise ValueError("orc_count_substeps failed")
    return counts, rows, iters, q, v, w
