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
                             target were ctrl + offset.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from paper_2502_08844_b300 import workloads as W

from . import oracle as O


def nrand(m) -> int:
    return 2 + 3 * m.nbody + m.nv + m.nu


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
    mass, ipos, inertia, arm = O.OracleModel(m).massprops()
    mass = mass.copy(); ipos = ipos.copy()
    if nb > 1:
        mass[1] += p[1]
    ipos += p[2:2 + 3 * nb].reshape(nb, 3)
    arm = arm + p[2 + 3 * nb:2 + 3 * nb + nv]
    return dataclasses.replace(
        m, body_geom_inertia=np.zeros(nb, np.int32), body_mass=mass, body_ipos=ipos, body_inertia=inertia,
        dof_armature=arm, dof_rotor=np.zeros((nv, 3)), pair_friction=m.pair_friction.astype(np.float64) * p[0],
        act_ctrllimited=np.zeros(nu, np.int32))


def controls(m, p, ctrl):
    """ctrl [..., nu] as the substituted model's actuators see it: clipped to a limited control
    range, then PD targets shifted by the calibration offsets."""
    p = np.asarray(p, np.float64)
    u = np.asarray(ctrl, np.float64).copy()
    lo, hi = m.act_ctrlrange[:, 0].astype(np.float64), m.act_ctrlrange[:, 1].astype(np.float64)
    lim = m.act_ctrllimited.astype(bool)
    u = np.where(lim, np.clip(u, lo, hi), u)
    cal = p[2 + 3 * m.nbody + m.nv:]
    return u + np.where(m.act_type == W.POSITION, cal, 0.0)
