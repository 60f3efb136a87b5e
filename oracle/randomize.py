"""What one environment's per-environment parameters mean, for the FP64 oracle (TEST
INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg import this
module.  The paper randomises ground friction, payload mass, link centres of mass, reflected
inertia and joint calibration offsets during training (App. B, "Domain Randomization").  The
CUDA path takes them as a per-environment parameter block (pg_step_dr); here an environment with
parameters p is defined as the nominal model with those values substituted, stepped by the
oracle's own physics:
  p[0]                       every pair's friction is multiplied by p[0];
  p[1]                       a point mass at body 1's centre of mass (mass + p[1], inertia about
                             the centre of mass unchanged);
  p[2 : 2 + 3 nbody]         each body's centre of mass moves by that offset (body frame),
                             inertia about the centre of mass unchanged;
  next nv                    armature added to each dof;
  next nu                    calibration offset: a PD actuator acts as if its (already clipped)
                             target were ctrl + offset;
  next nu                    kp scale s: a PD actuator's kp is kp (1 + s);
  next nu                    kd scale s: its kd is kd (1 + s);
  next nbody                 link mass scale s: body b's mass and its inertia about its centre
                             of mass are (1 + s) times the nominal (the payload is added after);
  next nv                    friction-loss scale s: a dof's joint friction loss is F (1 + s).
The PD gains, link masses and motor friction are the hand's additions (App. C.2).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from paper_2502_08844_b300 import workloads as W

from . import oracle as O


def nrand(m) -> int:
    return 2 + 4 * m.nbody + 2 * m.nv + 3 * m.nu


def rows(m) -> dict:
    """first row of each parameter group"""
    nb, nv, nu = m.nbody, m.nv, m.nu
    r = {"friction": 0, "payload": 1, "com": 2}
    r["armature"] = 2 + 3 * nb
    r["calibration"] = r["armature"] + nv
    r["kp"] = r["calibration"] + nu
    r["kd"] = r["kp"] + nu
    r["mass"] = r["kd"] + nu
    r["frictionloss"] = r["mass"] + nb
    return r


def nominal(m) -> np.ndarray:
    p = np.zeros(nrand(m))
    p[0] = 1.0
    return p


def substituted_model(m, p):
    """The model an environment with parameters p steps: explicit mass properties (the
    nominal model's own, derived from its geoms where it derives them) with the payload and
    centre-of-mass offsets applied, armature (rotor inertia included) plus p's, friction scaled.
    Actuator control limits are left to `controls`, which applies them before the offsets."""
    p = np.asarray(p, np.float64)
    nb, nv, nu = m.nbody, m.nv, m.nu
    R = rows(m)
    mass, ipos, inertia, arm = O.OracleModel(m).massprops()
    scale = 1.0 + p[R["mass"]:R["mass"] + nb]
    mass = mass * scale
    inertia = inertia * scale[:, None]
    ipos = ipos.copy()
    if nb > 1:
        mass[1] += p[1]
    ipos += p[2:2 + 3 * nb].reshape(nb, 3)
    arm = arm + p[R["armature"]:R["armature"] + nv]
    kp = m.act_kp.astype(np.float64) * (1.0 + p[R["kp"]:R["kp"] + nu])
    kd = m.act_kd.astype(np.float64) * (1.0 + p[R["kd"]:R["kd"] + nu])
    fl = m.dof_frictionloss
    if fl is not None:
        fl = fl.astype(np.float64) * (1.0 + p[R["frictionloss"]:R["frictionloss"] + nv])
    return dataclasses.replace(
        m, body_geom_inertia=np.zeros(nb, np.int32), body_mass=mass, body_ipos=ipos, body_inertia=inertia,
        dof_armature=arm, dof_rotor=np.zeros((nv, 3)), pair_friction=m.pair_friction.astype(np.float64) * p[0],
        act_ctrllimited=np.zeros(nu, np.int32), act_kp=kp, act_kd=kd, dof_frictionloss=fl)


def controls(m, p, ctrl):
    """ctrl [..., nu] as the substituted model's actuators see it: clipped to a limited control
    range, then PD targets shifted by the calibration offsets."""
    p = np.asarray(p, np.float64)
    u = np.asarray(ctrl, np.float64).copy()
    lo, hi = m.act_ctrlrange[:, 0].astype(np.float64), m.act_ctrlrange[:, 1].astype(np.float64)
    lim = m.act_ctrllimited.astype(bool)
    u = np.where(lim, np.clip(u, lo, hi), u)
    R = rows(m)
    cal = p[R["calibration"]:R["calibration"] + m.nu]
    return u + np.where(m.act_type == W.POSITION, cal, 0.0)
