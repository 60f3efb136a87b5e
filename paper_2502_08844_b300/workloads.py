"""Synthetic robot models and seeded inputs for the batched physics step.

This module only *describes* inputs: flat kinematic-tree arrays in level order
(the model format the library's compiler and the oracle both read) and the
seeded initial states and action sequences.  It contains none of the step's
arithmetic (no kinematics, dynamics, collision or solver code); both the CUDA
path and the FP64 oracle consume what it produces.

The paper's own workloads are MJCF robots from MuJoCo Menagerie and the DM
Control Suite (Sec. 2), which are not available here.  The models below stand
in for them at matching scale: a DM-Control-style cartpole, a Go1-like 12-DoF
quadruped with feet-only contacts (Sec. 4.2.1, App. B.2.3), a LEAP-like
16-DoF hand with a 7 cm cube (Sec. 4.3.1, App. C.2.2) and a G1-like 29-DoF
humanoid (Sec. 4.2.2).

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) with seed = config * 2**40 + env.
The k-th draw of a stream is mix(seed + (k + 1) * gamma), so any draw can be
generated independently; a draw becomes a double in [0, 1) from its top 53
bits, and every value handed to either path is first rounded to float32.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import numpy as np

# joint, geom, actuator and cone type codes (shared numbering of the model format)
FREE, HINGE, SLIDE = 0, 1, 2
PLANE, SPHERE, CAPSULE, BOX, HFIELD, CYLINDER, MESH = 0, 1, 2, 3, 4, 5, 6
MOTOR, POSITION = 0, 1
PYRAMIDAL, ELLIPTIC = 0, 1

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: np.ndarray, k: np.ndarray) -> np.ndarray:
    """k-th output (k >= 0) of the SplitMix64 stream started at `seed` (uint64, broadcast)."""
    with np.errstate(over="ignore"):
        z = np.asarray(seed, np.uint64) + (np.asarray(k, np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: np.ndarray, k: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of the k-th draw."""
    return (splitmix64(seed, k) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def env_seeds(config: int, n_envs: int, env0: int = 0) -> np.ndarray:
    return np.uint64(config) * np.uint64(1 << 40) + np.arange(env0, env0 + n_envs, dtype=np.uint64)


def _f32(x) -> np.ndarray:
    return np.asarray(x, dtype=np.float64).astype(np.float32)


# --------------------------------------------------------------------------------------
# model description
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Model:
    """Flat kinematic-tree arrays (body 0 is the world; parent[i] < i)."""

    name: str
    body_parent: np.ndarray      # [nbody] int32
    body_pos: np.ndarray         # [nbody,3] frame offset in the parent frame at q = 0
    body_quat: np.ndarray        # [nbody,4] (w,x,y,z)
    body_mass: np.ndarray        # [nbody]
    body_ipos: np.ndarray        # [nbody,3] centre of mass in the body frame
    body_inertia: np.ndarray     # [nbody,6] (xx,yy,zz,xy,xz,yz) about the COM, body axes
    body_geom_inertia: np.ndarray  # [nbody] int32: 1 = derive mass/COM/inertia from the body's geoms
    jnt_type: np.ndarray         # [njnt] int32 FREE/HINGE/SLIDE
    jnt_body: np.ndarray         # [njnt] int32 (joints grouped by body, in body order)
    jnt_pos: np.ndarray          # [njnt,3] anchor in the body frame
    jnt_axis: np.ndarray         # [njnt,3] axis in the body frame
    jnt_limited: np.ndarray      # [njnt] int32
    jnt_range: np.ndarray        # [njnt,2]
    dof_damping: np.ndarray      # [nv]
    dof_armature: np.ndarray     # [nv]
    dof_rotor: np.ndarray        # [nv,3] (gear ratio k_g, rotor mass m_r, rotor radius r_r); k_g = 0: none
    geom_type: np.ndarray        # [ngeom] int32
    geom_body: np.ndarray        # [ngeom] int32
    geom_pos: np.ndarray         # [ngeom,3]
    geom_quat: np.ndarray        # [ngeom,4]
    geom_size: np.ndarray        # [ngeom,3] sphere (r), capsule (r, half-length), box (half-sizes)
    geom_mass: np.ndarray        # [ngeom]
    pair_geom: np.ndarray        # [npair,2] int32 candidate contact pairs (geom1, geom2)
    pair_friction: np.ndarray    # [npair]
    pair_condim: np.ndarray      # [npair] int32: 1 (frictionless) or 3
    act_type: np.ndarray         # [nu] int32 MOTOR/POSITION
    act_jnt: np.ndarray          # [nu] int32 (hinge or slide joint)
    act_gear: np.ndarray         # [nu]
    act_kp: np.ndarray           # [nu]
    act_kd: np.ndarray           # [nu]
    act_ctrllimited: np.ndarray  # [nu] int32
    act_ctrlrange: np.ndarray    # [nu,2]
    timestep: float
    gravity: np.ndarray          # [3]
    iterations: int              # Newton iteration cap
    cone: int                    # PYRAMIDAL / ELLIPTIC
    impratio: float
    solref: np.ndarray           # [2] (timeconst, dampratio)
    solimp: np.ndarray           # [5] (d0, dwidth, width, mid, power)
    margin: float
    max_contacts: int            # cap on simultaneously active contacts
    n_substeps: int = 1          # physics substeps per control step for this workload
    default_ctrl: Optional[np.ndarray] = None  # [nu] e.g. the standing pose targets
    qpos_init: Optional[np.ndarray] = None     # [nq] reference initial configuration
    # the model's heightfield (HFIELD geoms, world-fixed): elevations in [0, 1], row i at
    # y = -hy + 2 hy i / (nrow - 1), column j at x = -hx + 2 hx j / (ncol - 1) of the geom frame;
    # the surface height is size[2] * elevation
    hfield: Optional[np.ndarray] = None        # [nrow, ncol] float32
    act_forcelimited: Optional[np.ndarray] = None   # [nu] int32: clip the actuator's force
    act_forcerange: Optional[np.ndarray] = None     # [nu, 2] (lo, hi)
    dof_frictionloss: Optional[np.ndarray] = None   # [nv] joint friction loss (a bound on its friction force)
    # convex meshes (MESH geoms): mesh k's vertices mesh_vert[mesh_vertadr[k] + i] (geom frame) and
    # outward counter-clockwise triangles mesh_face[mesh_faceadr[k] + f] (indices into its own
    # vertices) bounding their convex hull; geom_meshid[g] the mesh of a MESH geom, else -1
    mesh_vert: Optional[np.ndarray] = None          # [total vertices, 3] float32
    mesh_vertadr: Optional[np.ndarray] = None       # [nmesh] int32
    mesh_vertnum: Optional[np.ndarray] = None       # [nmesh] int32
    mesh_face: Optional[np.ndarray] = None          # [total faces, 3] int32
    mesh_faceadr: Optional[np.ndarray] = None       # [nmesh] int32
    mesh_facenum: Optional[np.ndarray] = None       # [nmesh] int32
    geom_meshid: Optional[np.ndarray] = None        # [ngeom] int32

    @property
    def nmesh(self) -> int:
        return 0 if self.mesh_vertadr is None else int(self.mesh_vertadr.shape[0])

    @property
    def nbody(self) -> int:
        return int(self.body_parent.shape[0])

    @property
    def njnt(self) -> int:
        return int(self.jnt_type.shape[0])

    @property
    def nq(self) -> int:
        return int(sum(7 if t == FREE else 1 for t in self.jnt_type))

    @property
    def nv(self) -> int:
        return int(sum(6 if t == FREE else 1 for t in self.jnt_type))

    @property
    def nu(self) -> int:
        return int(self.act_type.shape[0])

    @property
    def ngeom(self) -> int:
        return int(self.geom_type.shape[0])

    @property
    def npair(self) -> int:
        return int(self.pair_geom.shape[0])

    def jnt_qposadr(self) -> np.ndarray:
        adr, out = 0, []
        for t in self.jnt_type:
            out.append(adr)
            adr += 7 if t == FREE else 1
        return np.asarray(out, np.int32)

    def jnt_dofadr(self) -> np.ndarray:
        adr, out = 0, []
        for t in self.jnt_type:
            out.append(adr)
            adr += 6 if t == FREE else 1
        return np.asarray(out, np.int32)


class ModelBuilder:
    """Appends bodies, joints, geoms, pairs and actuators in level order."""

    def __init__(self, name: str):
        self.name = name
        self.bodies: List[dict] = [dict(parent=-1, pos=(0, 0, 0), quat=(1, 0, 0, 0), mass=0.0,
                                        ipos=(0, 0, 0), inertia=(0,) * 6, geom_inertia=0)]
        self.joints: List[dict] = []
        self.geoms: List[dict] = []
        self.pairs: List[dict] = []
        self.acts: List[dict] = []
        self.meshes: List[tuple] = []

    def body(self, parent: int, pos, quat=(1, 0, 0, 0), mass: float = 0.0, ipos=(0, 0, 0),
             inertia=(0,) * 6, geom_inertia: bool = True) -> int:
        assert 0 <= parent < len(self.bodies)
        self.bodies.append(dict(parent=parent, pos=pos, quat=quat, mass=mass, ipos=ipos,
                                inertia=inertia, geom_inertia=int(geom_inertia)))
        return len(self.bodies) - 1

    def joint(self, body: int, jtype: int, pos=(0, 0, 0), axis=(0, 0, 1), limited=False,
              range=(0.0, 0.0), damping=0.0, armature=0.0, rotor=(0.0, 0.0, 0.0), frictionloss=0.0) -> int:
        assert not self.joints or self.joints[-1]["body"] <= body, "joints must follow body order"
        self.joints.append(dict(body=body, type=jtype, pos=pos, axis=axis, limited=int(limited),
                                range=range, damping=damping, armature=armature, rotor=rotor,
                                frictionloss=frictionloss))
        return len(self.joints) - 1

    def geom(self, body: int, gtype: int, size, pos=(0, 0, 0), quat=(1, 0, 0, 0), mass=0.0, mesh: int = -1) -> int:
        s = list(size) + [0.0] * (3 - len(size))
        assert (gtype == MESH) == (mesh >= 0), "a MESH geom names its mesh (ModelBuilder.mesh)"
        self.geoms.append(dict(body=body, type=gtype, size=s, pos=pos, quat=quat, mass=mass, mesh=mesh))
        return len(self.geoms) - 1

    def mesh(self, vertices, faces) -> int:
        """a convex mesh: vertices [n, 3] and outward counter-clockwise triangles [f, 3] of their hull"""
        self.meshes.append((np.asarray(vertices, np.float64).reshape(-1, 3), np.asarray(faces, np.int64).reshape(-1, 3)))
        return len(self.meshes) - 1

    def pair(self, g1: int, g2: int, friction=1.0, condim=3) -> int:
        self.pairs.append(dict(g=(g1, g2), friction=friction, condim=condim))
        return len(self.pairs) - 1

    def actuator(self, jnt: int, atype: int, gear=1.0, kp=0.0, kd=0.0, ctrllimited=False,
                 ctrlrange=(0.0, 0.0), forcelimited=False, forcerange=(0.0, 0.0)) -> int:
        self.acts.append(dict(jnt=jnt, type=atype, gear=gear, kp=kp, kd=kd,
                              ctrllimited=int(ctrllimited), ctrlrange=ctrlrange,
                              forcelimited=int(forcelimited), forcerange=forcerange))
        return len(self.acts) - 1

    def build(self, *, timestep, gravity=(0, 0, -9.81), iterations=4, cone=PYRAMIDAL, impratio=1.0,
              solref=(0.02, 1.0), solimp=(0.9, 0.95, 0.001, 0.5, 2.0), margin=0.0,
              max_contacts=None, n_substeps=1, default_ctrl=None, qpos_init=None, hfield=None) -> Model:
        B, J, G = self.bodies, self.joints, self.geoms
        dof = []
        for j in J:
            n = 6 if j["type"] == FREE else 1
            dof += [j] * n
        maxpts = {(PLANE, SPHERE): 1, (PLANE, CAPSULE): 2, (PLANE, BOX): 4, (SPHERE, SPHERE): 1,
                  (SPHERE, CAPSULE): 1, (CAPSULE, CAPSULE): 1, (SPHERE, BOX): 1, (CAPSULE, BOX): 2,
                  (BOX, BOX): 4, (HFIELD, SPHERE): 1, (HFIELD, CAPSULE): 2, (PLANE, CYLINDER): 4,
                  (PLANE, MESH): 4, (HFIELD, BOX): 4, (HFIELD, MESH): 4}
        slots = sum(maxpts[(G[p["g"][0]]["type"], G[p["g"][1]]["type"])] for p in self.pairs)
        i32 = lambda x: np.asarray(x, np.int32)
        m = Model(
            name=self.name,
            body_parent=i32([b["parent"] for b in B]),
            body_pos=_f32([b["pos"] for b in B]).reshape(-1, 3),
            body_quat=_f32([b["quat"] for b in B]).reshape(-1, 4),
            body_mass=_f32([b["mass"] for b in B]),
            body_ipos=_f32([b["ipos"] for b in B]).reshape(-1, 3),
            body_inertia=_f32([b["inertia"] for b in B]).reshape(-1, 6),
            body_geom_inertia=i32([b["geom_inertia"] for b in B]),
            jnt_type=i32([j["type"] for j in J]),
            jnt_body=i32([j["body"] for j in J]),
            jnt_pos=_f32([j["pos"] for j in J]).reshape(-1, 3),
            jnt_axis=_f32([j["axis"] for j in J]).reshape(-1, 3),
            jnt_limited=i32([j["limited"] for j in J]),
            jnt_range=_f32([j["range"] for j in J]).reshape(-1, 2),
            dof_damping=_f32([j["damping"] for j in dof]),
            dof_armature=_f32([j["armature"] for j in dof]),
            dof_rotor=_f32([j["rotor"] for j in dof]).reshape(-1, 3),
            geom_type=i32([g["type"] for g in G]),
            geom_body=i32([g["body"] for g in G]),
            geom_pos=_f32([g["pos"] for g in G]).reshape(-1, 3),
            geom_quat=_f32([g["quat"] for g in G]).reshape(-1, 4),
            geom_size=_f32([g["size"] for g in G]).reshape(-1, 3),
            geom_mass=_f32([g["mass"] for g in G]),
            pair_geom=i32([p["g"] for p in self.pairs]).reshape(-1, 2),
            pair_friction=_f32([p["friction"] for p in self.pairs]),
            pair_condim=i32([p["condim"] for p in self.pairs]),
            act_type=i32([a["type"] for a in self.acts]),
            act_jnt=i32([a["jnt"] for a in self.acts]),
            act_gear=_f32([a["gear"] for a in self.acts]),
            act_kp=_f32([a["kp"] for a in self.acts]),
            act_kd=_f32([a["kd"] for a in self.acts]),
            act_ctrllimited=i32([a["ctrllimited"] for a in self.acts]),
            act_ctrlrange=_f32([a["ctrlrange"] for a in self.acts]).reshape(-1, 2),
            timestep=float(np.float32(timestep)),
            gravity=_f32(gravity),
            iterations=int(iterations),
            cone=int(cone),
            impratio=float(np.float32(impratio)),
            solref=_f32(solref),
            solimp=_f32(solimp),
            margin=float(np.float32(margin)),
            max_contacts=int(slots if max_contacts is None else max_contacts),
            n_substeps=int(n_substeps),
            default_ctrl=None if default_ctrl is None else _f32(default_ctrl),
            qpos_init=None if qpos_init is None else _f32(qpos_init),
            hfield=None if hfield is None else _f32(hfield),
        )
        if any(j["frictionloss"] > 0 for j in J):
            m.dof_frictionloss = _f32([j["frictionloss"] for j in dof])
        if self.meshes:
            nv_ = [v.shape[0] for v, _ in self.meshes]
            nf_ = [f.shape[0] for _, f in self.meshes]
            m.mesh_vert = _f32(np.concatenate([v for v, _ in self.meshes]))
            m.mesh_vertadr = i32(np.concatenate([[0], np.cumsum(nv_)[:-1]]))
            m.mesh_vertnum = i32(nv_)
            m.mesh_face = i32(np.concatenate([f for _, f in self.meshes]))
            m.mesh_faceadr = i32(np.concatenate([[0], np.cumsum(nf_)[:-1]]))
            m.mesh_facenum = i32(nf_)
            m.geom_meshid = i32([g["mesh"] for g in G])
        if any(a["forcelimited"] for a in self.acts):
            m.act_forcelimited = i32([a["forcelimited"] for a in self.acts])
            m.act_forcerange = _f32([a["forcerange"] for a in self.acts]).reshape(-1, 2)
        return m


def _axis_quat(axis, angle):
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    return (math.cos(angle / 2),) + tuple(a * math.sin(angle / 2))


# --------------------------------------------------------------------------------------
# the synthetic models
# --------------------------------------------------------------------------------------

def cartpole() -> Model:
    """Cart on a slider (box 0.4x0.2x0.1 m, 1 kg, damping 0.1) carrying a hinged pole
    (capsule 1.0 m, radius 0.05 m, 0.1 kg); motor with gear 10 on the slider; dt 0.01 s.
    q = 0 is the pole upright.  No contacts and no limits."""
    b = ModelBuilder("cartpole")
    cart = b.body(0, (0, 0, 0))
    b.joint(cart, SLIDE, axis=(1, 0, 0), damping=0.1)
    b.geom(cart, BOX, (0.2, 0.1, 0.05), mass=1.0)
    pole = b.body(cart, (0, 0, 0))
    b.joint(pole, HINGE, axis=(0, 1, 0))
    b.geom(pole, CAPSULE, (0.05, 0.5), pos=(0, 0, 0.5), mass=0.1)
    b.actuator(0, MOTOR, gear=10.0, ctrllimited=True, ctrlrange=(-1.0, 1.0))
    return b.build(timestep=0.01, iterations=1, n_substeps=1, qpos_init=(0.0, 0.0))


QUAD_HIP = ((0.19, 0.05), (0.19, -0.05), (-0.19, 0.05), (-0.19, -0.05))
QUAD_STAND = (0.0, 0.9, -1.8)       # (abduction, flexion, knee) per leg
QUAD_LINK = 0.2
QUAD_FOOT_R = 0.02


def quadruped_standing_height() -> float:
    """Torso height with every foot 1 mm above the plane in the standing pose: the hip is
    at the torso origin height and thigh + calf make a closed 'V' (0.9 rad and -1.8 rad)."""
    th, kn = QUAD_STAND[1], QUAD_STAND[2]
    drop = QUAD_LINK * math.cos(th) + QUAD_LINK * math.cos(th + kn)
    return drop + QUAD_FOOT_R + 0.001


def quadruped() -> Model:
    """Floating-base quadruped: torso box 0.38x0.1x0.1 m, 5 kg; per leg an abduction (x) and a
    flexion (y) hinge at the hip, thigh capsule 0.2 m r 0.02 0.6 kg, knee (y) hinge, calf capsule
    0.2 m r 0.02 0.15 kg and a massless r 0.02 foot sphere.  Feet-only foot/plane contacts,
    friction 1, pyramidal cone; PD kp 35 kd 0.5; dt 0.004 s, 5 substeps, Newton cap 4."""
    b = ModelBuilder("quadruped")
    floor = b.geom(0, PLANE, (0, 0, 0))
    z0 = quadruped_standing_height()
    torso = b.body(0, (0, 0, z0))
    b.joint(torso, FREE)
    b.geom(torso, BOX, (0.19, 0.05, 0.05), mass=5.0)
    thighs, calves, feet = [], [], []
    for hx, hy in QUAD_HIP:
        t = b.body(torso, (hx, hy, 0.0))
        b.joint(t, HINGE, axis=(1, 0, 0), limited=True, range=(-1.0, 1.0))
        b.joint(t, HINGE, axis=(0, 1, 0), limited=True, range=(-1.5, 1.5))
        b.geom(t, CAPSULE, (QUAD_FOOT_R, QUAD_LINK / 2), pos=(0, 0, -QUAD_LINK / 2), mass=0.6)
        thighs.append(t)
    for t in thighs:
        c = b.body(t, (0, 0, -QUAD_LINK))
        b.joint(c, HINGE, axis=(0, 1, 0), limited=True, range=(-2.7, -0.9))
        b.geom(c, CAPSULE, (QUAD_FOOT_R, QUAD_LINK / 2), pos=(0, 0, -QUAD_LINK / 2), mass=0.15)
        feet.append(b.geom(c, SPHERE, (QUAD_FOOT_R,), pos=(0, 0, -QUAD_LINK), mass=0.0))
        calves.append(c)
    for f in feet:
        b.pair(floor, f, friction=1.0, condim=3)
    # actuators in joint order: 4 x (abduction, flexion) then 4 x knee
    for j in range(1, 13):
        b.actuator(j, POSITION, kp=35.0, kd=0.5)
    stand = [QUAD_STAND[0], QUAD_STAND[1]] * 4 + [QUAD_STAND[2]] * 4
    qpos = [0.0, 0.0, z0, 1.0, 0.0, 0.0, 0.0] + stand
    return b.build(timestep=0.004, iterations=4, cone=PYRAMIDAL, n_substeps=5,
                   default_ctrl=stand, qpos_init=qpos)


_ROT_Z_TO_Y = (math.cos(-math.pi / 4), math.sin(-math.pi / 4), 0.0, 0.0)   # capsule axis along +y
_ROT_Z_TO_X = (math.cos(math.pi / 4), 0.0, math.sin(math.pi / 4), 0.0)     # capsule axis along +x

# LEAP-hand style rotor (App. C.2.2): gear ratio 288.35, rotor 2.0 g, radius 4.12 mm
HAND_ROTOR = (288.35, 2.0e-3, 4.12e-3)
HAND_PHALANX = ((0.05, 0.05), (0.04, 0.04), (0.035, 0.03), (0.03, 0.02))   # (length, mass)
HAND_CUBE = 0.07
HAND_CUBE_Y = 0.025   # cube centre towards the finger roots: curled fingers reach its +y face


def hand(max_contacts: int = 20, cone: int = PYRAMIDAL, frictionloss: float = 0.0) -> Model:
    """Fixed-base 16-hinge hand with a free 7 cm cube (LEAP-like, App. C.2).  World-fixed palm box
    0.12x0.10x0.02 m with its top face at z = 0; 4 fingers rooted on the palm's +y edge, each a
    chain of 4 capsule phalanges (r 0.01; 0.05/0.04/0.035/0.03 m, 0.05/0.04/0.03/0.02 kg) with
    joints abduction (z) then 3 flexions (x), and a fingertip sphere r 0.012.  Reflected rotor
    inertia on every dof from the paper's servo numbers.  The cube rests on the palm near the
    finger roots (centre y = 0.025).  Contacts: fingertip spheres and the
    capsules of the last three phalanges against the cube, cube against palm; at most 20 active,
    friction 1, pyramidal cone.  PD kp 3 kd 0.1; dt 5 ms, 10 substeps, Newton cap 6.
    `frictionloss` > 0 gives every hinge that joint friction loss (App. C.2.2 sets it to a tenth of
    the servo's maximum torque)."""
    b = ModelBuilder("hand")
    palm = b.geom(0, BOX, (0.06, 0.05, 0.01), pos=(0, 0, -0.01))
    tips, caps = [], []
    for i in range(4):
        parent, pos = 0, (-0.045 + 0.03 * i, 0.05, 0.0)
        for s, (L, m) in enumerate(HAND_PHALANX):
            link = b.body(parent, pos)
            if s == 0:
                b.joint(link, HINGE, axis=(0, 0, 1), limited=True, range=(-0.5, 0.5), rotor=HAND_ROTOR,
                        frictionloss=frictionloss)
            else:
                b.joint(link, HINGE, axis=(1, 0, 0), limited=True, range=(-0.3, 1.6), rotor=HAND_ROTOR,
                        frictionloss=frictionloss)
            g = b.geom(link, CAPSULE, (0.01, L / 2), pos=(0, L / 2, 0), quat=_ROT_Z_TO_Y, mass=m)
            if s > 0:
                caps.append(g)
            if s == 3:
                tips.append(b.geom(link, SPHERE, (0.012,), pos=(0, L, 0), mass=0.0))
            parent, pos = link, (0, L, 0)
    cube = b.body(0, (0, HAND_CUBE_Y, HAND_CUBE / 2))
    b.joint(cube, FREE)
    cg = b.geom(cube, BOX, (HAND_CUBE / 2,) * 3, mass=0.1)
    for t in tips:
        b.pair(t, cg, friction=1.0, condim=3)
    for g in caps:
        b.pair(g, cg, friction=1.0, condim=3)
    b.pair(palm, cg, friction=1.0, condim=3)
    for j in range(16):   # targets are drawn within the joint's range
        b.actuator(j, POSITION, kp=3.0, kd=0.1, ctrlrange=(-0.5, 0.5) if j % 4 == 0 else (-0.3, 1.6))
    qpos = [0.0] * 16 + [0.0, HAND_CUBE_Y, HAND_CUBE / 2, 1.0, 0.0, 0.0, 0.0]
    m = b.build(timestep=0.005, iterations=6, cone=cone, n_substeps=10, max_contacts=max_contacts, qpos_init=qpos)
    if cone == ELLIPTIC:
        m.name = "hand_elliptic"
    return m


def hand_elliptic() -> Model:
    """The hand with the elliptic friction cone (the workload's other cone option)."""
    return hand(cone=ELLIPTIC)


def humanoid() -> Model:
    """Floating-base 29-hinge humanoid (G1-like, Sec. 4.2.2): pelvis with a free joint; waist
    (3 hinges) carrying the torso and two 7-hinge arms (shoulder 3, elbow, wrist 3); two 6-hinge
    legs (hip 3, knee, ankle 2) with box feet 0.2x0.08x0.03 m.  Capsule links 0.08-0.36 m, masses
    scaled to 35 kg.  Contacts: each foot box against the plane (<= 4 points), each hand capsule
    against the torso capsule; friction 1, pyramidal.  PD on every hinge (legs/waist kp 60 kd 2,
    arms kp 20 kd 0.5), armature 0.01; dt 4 ms, 5 substeps, Newton cap 4."""
    raw = {"pelvis": 6.0, "torso": 12.0, "thigh": 4.5, "shin": 2.5, "foot": 0.8, "upper": 1.5, "fore": 1.0,
           "hand": 0.4}
    total = raw["pelvis"] + raw["torso"] + 2 * (raw["thigh"] + raw["shin"] + raw["foot"] + raw["upper"] + raw["fore"]
                                                 + raw["hand"])
    s = 35.0 / total
    ms = {k: v * s for k, v in raw.items()}
    b = ModelBuilder("humanoid")
    floor = b.geom(0, PLANE, (0, 0, 0))
    z0 = 0.05 + 0.4 + 0.4 + 0.05 + 0.015 + 0.001
    pelvis = b.body(0, (0, 0, z0))
    b.joint(pelvis, FREE)
    b.geom(pelvis, CAPSULE, (0.07, 0.08), quat=_ROT_Z_TO_Y, mass=ms["pelvis"])
    torso = b.body(pelvis, (0, 0, 0.1))
    arm = dict(armature=0.01, limited=True)
    for ax in ((0, 0, 1), (1, 0, 0), (0, 1, 0)):
        b.joint(torso, HINGE, axis=ax, range=(-0.5, 0.5), **arm)
    torso_g = b.geom(torso, CAPSULE, (0.1, 0.12), pos=(0, 0, 0.2), mass=ms["torso"])
    hips, shoulders = [], []
    for side in (1, -1):
        hips.append(b.body(pelvis, (0, 0.1 * side, -0.05)))
    for side in (1, -1):
        shoulders.append(b.body(torso, (0, 0.22 * side, 0.3)))
    knees, ankles, feet = [], [], []
    for h_ in hips:
        b.joint(h_, HINGE, axis=(1, 0, 0), range=(-0.5, 0.5), **arm)
        b.joint(h_, HINGE, axis=(0, 0, 1), range=(-0.5, 0.5), **arm)
        b.joint(h_, HINGE, axis=(0, 1, 0), range=(-1.5, 1.0), **arm)
        b.geom(h_, CAPSULE, (0.06, 0.18), pos=(0, 0, -0.2), mass=ms["thigh"])
    elbows, wrists, hands = [], [], []
    for sh in shoulders:
        b.joint(sh, HINGE, axis=(0, 1, 0), range=(-1.5, 1.5), **arm)
        b.joint(sh, HINGE, axis=(1, 0, 0), range=(-1.5, 1.5), **arm)
        b.joint(sh, HINGE, axis=(0, 0, 1), range=(-1.5, 1.5), **arm)
        b.geom(sh, CAPSULE, (0.04, 0.12), pos=(0, 0, -0.14), mass=ms["upper"])
    for h_ in hips:
        k = b.body(h_, (0, 0, -0.4))
        b.joint(k, HINGE, axis=(0, 1, 0), range=(-0.1, 2.3), **arm)
        b.geom(k, CAPSULE, (0.05, 0.18), pos=(0, 0, -0.2), mass=ms["shin"])
        knees.append(k)
    for sh in shoulders:
        e = b.body(sh, (0, 0, -0.28))
        b.joint(e, HINGE, axis=(0, 1, 0), range=(-2.5, 0.0), **arm)
        b.geom(e, CAPSULE, (0.035, 0.1), pos=(0, 0, -0.12), mass=ms["fore"])
        elbows.append(e)
    for k in knees:
        a = b.body(k, (0, 0, -0.4))
        b.joint(a, HINGE, axis=(0, 1, 0), range=(-0.8, 0.8), **arm)
        b.joint(a, HINGE, axis=(1, 0, 0), range=(-0.4, 0.4), **arm)
        feet.append(b.geom(a, BOX, (0.1, 0.04, 0.015), pos=(0.03, 0, -0.05), mass=ms["foot"]))
        ankles.append(a)
    for e in elbows:
        w = b.body(e, (0, 0, -0.25))
        b.joint(w, HINGE, axis=(0, 0, 1), range=(-0.8, 0.8), **arm)
        b.joint(w, HINGE, axis=(0, 1, 0), range=(-0.8, 0.8), **arm)
        b.joint(w, HINGE, axis=(1, 0, 0), range=(-0.8, 0.8), **arm)
        hands.append(b.geom(w, CAPSULE, (0.04, 0.04), pos=(0, 0, -0.06), mass=ms["hand"]))
        wrists.append(w)
    for f in feet:
        b.pair(floor, f, friction=1.0, condim=3)
    for hg in hands:
        b.pair(torso_g, hg, friction=1.0, condim=3)
    # PD on every hinge, in joint order; the first 3 hinges (waist) and the legs are stiffer
    legs = set()
    for j in range(1, b_njnt(b)):
        body = b.joints[j]["body"]
        if body in hips or body in knees or body in ankles or body == torso:
            legs.add(j)
    for j in range(1, b_njnt(b)):
        if j in legs:
            b.actuator(j, POSITION, kp=60.0, kd=2.0)
        else:
            b.actuator(j, POSITION, kp=20.0, kd=0.5)
    nh = b_njnt(b) - 1
    qpos = [0.0, 0.0, z0, 1.0, 0.0, 0.0, 0.0] + [0.0] * nh
    return b.build(timestep=0.004, iterations=4, cone=PYRAMIDAL, n_substeps=5, max_contacts=16,
                   default_ctrl=[0.0] * nh, qpos_init=qpos)


def b_njnt(b: ModelBuilder) -> int:
    return len(b.joints)


MODELS = {"cartpole": cartpole, "quadruped": quadruped, "hand": hand, "hand_elliptic": hand_elliptic, "humanoid": humanoid}


def perlin_terrain(nrow: int, ncol: int, cells: int, seed: int) -> np.ndarray:
    """Elevations [nrow, ncol] in [0, 1] of 2-D gradient noise (Perlin's construction: unit
    gradients drawn at the corners of a cells x cells lattice, the smoothstep 6t^5 - 15t^4 + 10t^3
    blend of the corners' dot products), rescaled to span [0, 1].  Seeded, deterministic."""
    g = uniform01(np.full((cells + 1) * (cells + 1), np.uint64(seed)), np.arange((cells + 1) ** 2, dtype=np.uint64))
    ang = (2.0 * np.pi * g).reshape(cells + 1, cells + 1)
    gx, gy = np.cos(ang), np.sin(ang)
    y = np.linspace(0.0, cells, nrow, endpoint=False) + 0.5 * cells / nrow
    x = np.linspace(0.0, cells, ncol, endpoint=False) + 0.5 * cells / ncol
    Y, X = np.meshgrid(y, x, indexing="ij")
    i0, j0 = np.floor(Y).astype(int), np.floor(X).astype(int)
    fy, fx = Y - i0, X - j0
    fade = lambda t: t * t * t * (t * (6.0 * t - 15.0) + 10.0)

    def corner(di, dj):
        return gx[i0 + di, j0 + dj] * (fx - dj) + gy[i0 + di, j0 + dj] * (fy - di)

    u, v = fade(fx), fade(fy)
    top = corner(0, 0) + u * (corner(0, 1) - corner(0, 0))
    bot = corner(1, 0) + u * (corner(1, 1) - corner(1, 0))
    n = top + v * (bot - top)
    return _f32((n - n.min()) / (n.max() - n.min()))


ROUGH_HALF = 4.0       # the terrain spans 8 m x 8 m
ROUGH_SAMPLES = 81     # 0.1 m cells
ROUGH_HEIGHT = 0.06    # 6 cm between the lowest and the highest point


def quadruped_rough() -> Model:
    """The quadruped on rough terrain: the floor plane replaced by an 8 m x 8 m heightfield of
    gradient noise (81 x 81 samples, 0.1 m cells, 6 cm relief, 0.5 m noise lattice), the rough-terrain setting of the
    locomotion fine-tuning (App. B, "Finetuning").  The base starts high enough that no foot
    starts below the terrain."""
    m = quadruped()
    m.name = "quadruped_rough"
    hf = perlin_terrain(ROUGH_SAMPLES, ROUGH_SAMPLES, 16, seed=7)
    m.geom_type = m.geom_type.copy(); m.geom_size = m.geom_size.copy()
    m.geom_type[0] = HFIELD
    m.geom_size[0] = _f32([ROUGH_HALF, ROUGH_HALF, ROUGH_HEIGHT])
    m.hfield = hf
    m.qpos_init = m.qpos_init.copy()
    m.qpos_init[2] += np.float32(ROUGH_HEIGHT * float(hf.max()))
    m.body_pos = m.body_pos.copy()
    m.body_pos[1, 2] = m.qpos_init[2]
    return m


MODELS["quadruped_rough"] = quadruped_rough


def humanoid_rough() -> Model:
    """The humanoid on the rough terrain of quadruped_rough (the humanoids' training follows the
    quadruped's fine-tuning, Sec. 4.2.2): its floor plane replaced by the 8 m x 8 m heightfield, so
    each box foot meets the terrain as a solid (heightfield-box pairs).  The pelvis starts raised
    by the terrain's highest point."""
    m = humanoid()
    m.name = "humanoid_rough"
    hf = perlin_terrain(ROUGH_SAMPLES, ROUGH_SAMPLES, 16, seed=7)
    m.geom_type = m.geom_type.copy(); m.geom_size = m.geom_size.copy()
    assert m.geom_type[0] == PLANE
    m.geom_type[0] = HFIELD
    m.geom_size[0] = _f32([ROUGH_HALF, ROUGH_HALF, ROUGH_HEIGHT])
    m.hfield = hf
    m.qpos_init = m.qpos_init.copy()
    m.qpos_init[2] += np.float32(ROUGH_HEIGHT * float(hf.max()))
    m.body_pos = m.body_pos.copy()
    m.body_pos[1, 2] = m.qpos_init[2]
    return m


MODELS["humanoid_rough"] = humanoid_rough


def convex_hull(seed: int, n_points: int, radii) -> tuple:
    """A seeded convex polytope: n_points drawn uniformly on the ellipsoid of semi-axes `radii`
    (directions from normalised Gaussian pairs of draws, Box-Muller), their convex hull
    (scipy.spatial.ConvexHull) with only its vertices kept and every triangle turned outward
    (counter-clockwise seen from outside).  Returns (vertices [n, 3], faces [f, 3])."""
    from scipy.spatial import ConvexHull
    k = np.arange(4 * n_points, dtype=np.uint64)
    u = uniform01(np.full(k.shape, np.uint64(seed)), k).reshape(n_points, 4)
    r = np.sqrt(-2.0 * np.log(1.0 - u[:, :2]))
    g = np.stack([r[:, 0] * np.cos(2 * np.pi * u[:, 2]), r[:, 0] * np.sin(2 * np.pi * u[:, 2]),
                  r[:, 1] * np.cos(2 * np.pi * u[:, 3])], axis=1)
    pts = g / np.linalg.norm(g, axis=1, keepdims=True) * np.asarray(radii, np.float64)
    pts = _f32(pts).astype(np.float64)            # the float32 vertices the library receives
    hull = ConvexHull(pts)
    keep = np.sort(hull.vertices)
    remap = -np.ones(n_points, np.int64)
    remap[keep] = np.arange(keep.size)
    faces = []
    for tri, eq in zip(hull.simplices, hull.equations):
        a, b, c = pts[tri]
        if np.dot(np.cross(b - a, c - a), eq[:3]) < 0:
            tri = tri[[0, 2, 1]]
        faces.append(remap[tri])
    return pts[keep], np.asarray(faces, np.int64)


def hulls() -> Model:
    """Convex rocks: three seeded convex hulls (12, 16 and 20 points on ellipsoids of 4-8 cm
    semi-axes, 0.2-0.4 kg, uniform density) as free bodies, the first two 14 cm above a plane and
    the third 20 cm above a 2 m x 2 m heightfield of gradient noise (41 x 41 samples, 5 cm cells, 4 cm
    relief) beside it; plane-mesh and heightfield-mesh pairs (4 points each), friction 0.8,
    pyramidal; dt 2 ms, 4 substeps, Newton cap 6."""
    b = ModelBuilder("hulls")
    floor = b.geom(0, PLANE, (0, 0, 0))
    terrain = b.geom(0, HFIELD, (1.0, 1.0, 0.04), pos=(3.0, 0, 0))
    shapes = [(101, 12, (0.08, 0.06, 0.05), 0.3, (0.0, 0.0, 0.14)), (102, 16, (0.05, 0.07, 0.04), 0.2, (0.4, 0.1, 0.14)),
              (103, 20, (0.06, 0.06, 0.08), 0.4, (3.1, -0.2, 0.2))]
    qpos = []
    for seed, npts, radii, mass, pos in shapes:
        v, f = convex_hull(seed, npts, radii)
        mk = b.mesh(v, f)
        body = b.body(0, pos)
        b.joint(body, FREE)
        g = b.geom(body, MESH, (0, 0, 0), mass=mass, mesh=mk)
        b.pair(terrain if pos[0] > 2.0 else floor, g, friction=0.8, condim=3)
        qpos += list(pos) + [1.0, 0.0, 0.0, 0.0]
    hf = perlin_terrain(41, 41, 8, seed=11)
    return b.build(timestep=0.002, iterations=6, n_substeps=4, qpos_init=qpos, hfield=hf)


MODELS["hulls"] = hulls


# --------------------------------------------------------------------------------------
# pixel observations: a camera, a light and the geoms' colours (configuration only)
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Scene:
    """What pg_render draws: a pinhole camera, one directional light and per-geom albedo
    (a negative first component hides a geom)."""

    cam_pos: tuple
    cam_lookat: tuple
    cam_up: tuple
    fovy_deg: float
    width: int
    height: int
    light_dir: tuple
    ambient: float
    diffuse: float
    background: tuple
    geom_rgb: np.ndarray      # [ngeom, 3] float32


def cartpole_pixels() -> Model:
    """The cartpole with a floor plane 6 cm under the cart's centre for its pixel
    observations (the floor pairs with nothing: the physics is the cartpole's)."""
    m = cartpole()
    m.name = "cartpole_pixels"
    m.geom_type = np.concatenate([m.geom_type, np.array([PLANE], np.int32)])
    m.geom_body = np.concatenate([m.geom_body, np.array([0], np.int32)])
    m.geom_pos = np.concatenate([m.geom_pos, _f32([[0, 0, -0.06]])])
    m.geom_quat = np.concatenate([m.geom_quat, _f32([[1, 0, 0, 0]])])
    m.geom_size = np.concatenate([m.geom_size, _f32([[0, 0, 0]])])
    m.geom_mass = np.concatenate([m.geom_mass, _f32([0])])
    return m


MODELS["cartpole_pixels"] = cartpole_pixels


def cartpole_scene(width: int = 64, height: int = 64) -> Scene:
    """The 64 x 64 pixel observation of the cartpole (the resolution of the paper's pixel
    policies): camera 3 m in front, looking at the pole's middle, light from above and behind."""
    return Scene(cam_pos=(0.0, -3.0, 0.7), cam_lookat=(0.0, 0.0, 0.4), cam_up=(0.0, 0.0, 1.0), fovy_deg=45.0,
                 width=width, height=height, light_dir=(0.35, 0.45, -1.0), ambient=0.25, diffuse=0.75,
                 background=(0.45, 0.6, 0.85),
                 geom_rgb=_f32([[0.2, 0.35, 0.85], [0.9, 0.55, 0.15], [0.6, 0.6, 0.6]]))


def quadruped_scene(width: int = 64, height: int = 64) -> Scene:
    """The quadruped from the front-left, every geom drawn (planes, boxes, capsules, spheres)."""
    m = quadruped()
    rgb = np.tile(_f32([[0.75, 0.45, 0.2]]), (m.ngeom, 1))
    rgb[0] = (0.55, 0.6, 0.55)                     # floor
    rgb[1] = (0.2, 0.3, 0.8)                       # torso
    rgb[m.geom_type == SPHERE] = (0.1, 0.1, 0.1)   # feet
    return Scene(cam_pos=(0.9, -1.1, 0.6), cam_lookat=(0.0, 0.0, 0.2), cam_up=(0.0, 0.0, 1.0), fovy_deg=50.0,
                 width=width, height=height, light_dir=(-0.3, 0.5, -1.0), ambient=0.3, diffuse=0.7,
                 background=(0.5, 0.65, 0.9), geom_rgb=_f32(rgb))


# --------------------------------------------------------------------------------------
# locomotion task around the step (configuration only: which geoms are feet, the weights of
# the reward table's terms, the action mapping; the arithmetic lives in the kernels and, for
# tests, in the oracle)
# --------------------------------------------------------------------------------------

ABSOLUTE, RELATIVE = 0, 1
# reward terms in the order of the C ABI's PG_R_* list
TERMS = ("lin_vel", "ang_vel", "air_time", "clearance", "slip", "orientation", "torque", "joint_pos",
         "action_rate", "energy", "pose", "termination", "stand_still", "lin_z", "ang_xy")
# joystick command ranges (vx, vy, wz) of the first joystick training stage (App. B, "Finetuning")
COMMAND_RANGE = (1.5, 0.8, 1.2)


@dataclasses.dataclass
class Task:
    """A locomotion task: the action mapping, the feet and the reward table's weights."""

    action_mode: int             # ABSOLUTE (q_default + scale a) or RELATIVE (q_des_prev + scale a)
    action_scale: float
    q_default: np.ndarray        # [nu] float32
    foot_geom: np.ndarray        # [nfeet] int32 sphere geoms
    contact_height: float        # a foot touches the ground below this height of its lowest point
    clearance_height: float      # desired swing height
    sigma_lin_vel: float
    sigma_ang_vel: float
    air_time_min: float
    air_time_max: float
    weight: np.ndarray           # [len(TERMS)] float32
    episode_length: int

    @property
    def nfeet(self) -> int:
        return int(self.foot_geom.shape[0])


# Weights of the quadruped joystick task. The paper prints the reward table without its
# coefficients; these are this workload's own choice (tracking rewards positive, penalties
# negative), not the paper's.
QUAD_TASK_WEIGHTS = {"lin_vel": 1.0, "ang_vel": 0.5, "air_time": 0.1, "clearance": -2.0, "slip": -0.1,
                     "orientation": -5.0, "torque": -2e-4, "joint_pos": -0.05, "action_rate": -0.01,
                     "energy": -1e-3, "pose": 0.5, "termination": -1.0, "stand_still": -0.5, "lin_z": -0.5,
                     "ang_xy": -0.05}


def quadruped_task(action_mode: int = ABSOLUTE, episode_length: int = 1000, weights=None) -> Task:
    """Joystick locomotion task of the quadruped: absolute targets around the standing pose
    (action scale 0.3 rad), the four foot spheres as feet."""
    m = quadruped()
    feet = np.array([g for g in range(m.ngeom) if m.geom_type[g] == SPHERE], np.int32)
    w = dict(QUAD_TASK_WEIGHTS)
    if weights:
        w.update(weights)
    return Task(action_mode=action_mode, action_scale=0.3, q_default=_f32(m.default_ctrl), foot_geom=feet,
                contact_height=0.002, clearance_height=0.08, sigma_lin_vel=0.25, sigma_ang_vel=0.25,
                air_time_min=0.1, air_time_max=0.5, weight=_f32([w[k] for k in TERMS]),
                episode_length=int(episode_length))


def commands(config: int, n_envs: int, env0: int = 0, draw: int = 0) -> np.ndarray:
    """Joystick commands [N, 3] (vx, vy, wz) float32, uniform in +-COMMAND_RANGE; draw index
    2^32 + 3 draw + k of each env's stream."""
    seeds = env_seeds(config, n_envs, env0)[:, None]
    k = np.uint64(1 << 32) + np.uint64(3 * draw) + np.arange(3, dtype=np.uint64)[None, :]
    u = uniform01(seeds, k)
    return _f32((2.0 * u - 1.0) * np.array(COMMAND_RANGE)[None, :])


def randomized_params(m: Model, config: int, n_envs: int, env0: int = 0) -> np.ndarray:
    """Per-environment physical parameters [N, 2 + 4 nbody + 2 nv + 3 nu] float32 in the layout
    of pg_step_dr: friction scale U[0.6, 1.4], payload U[0, 2] kg on body 1, centre-of-mass
    offsets U(+-2 cm), added armature U[0, 0.01] kg m^2, calibration offsets U(+-0.05) rad, kp and
    kd scales U(+-20 %), link mass scales U(+-10 %), friction-loss scales U(+-50 %); draw index
    2^34 + k of each env's stream."""
    nb, nv, nu = m.nbody, m.nv, m.nu
    k = 2 + 4 * nb + 2 * nv + 3 * nu
    seeds = env_seeds(config, n_envs, env0)[:, None]
    u = uniform01(seeds, np.uint64(1 << 34) + np.arange(k, dtype=np.uint64)[None, :])
    sym = 2.0 * u - 1.0
    p = np.zeros((n_envs, k))
    arm, cal = 2 + 3 * nb, 2 + 3 * nb + nv
    kp, kd, ms, fl = cal + nu, cal + 2 * nu, cal + 3 * nu, cal + 3 * nu + nb
    p[:, 0] = 0.6 + 0.8 * u[:, 0]
    p[:, 1] = 2.0 * u[:, 1]
    p[:, 2:arm] = 0.02 * sym[:, 2:arm]
    p[:, arm:cal] = 0.01 * u[:, arm:cal]
    p[:, cal:kp] = 0.05 * sym[:, cal:kp]
    p[:, kp:ms] = 0.2 * sym[:, kp:ms]
    p[:, ms:fl] = 0.1 * sym[:, ms:fl]
    p[:, fl:] = 0.5 * sym[:, fl:]
    return _f32(p)


def policy_actions(m: Model, config: int, n_envs: int, t0: int, n_steps: int, env0: int = 0) -> np.ndarray:
    """Policy outputs [n_steps, N, nu] float32, uniform in [-1, 1]; draw index
    2^33 + t nu + j of each env's stream."""
    seeds = env_seeds(config, n_envs, env0)[None, :, None]
    nu = m.nu
    t = np.arange(t0, t0 + n_steps, dtype=np.uint64)[:, None, None]
    j = np.arange(nu, dtype=np.uint64)[None, None, :]
    u = uniform01(seeds, np.uint64(1 << 33) + t * np.uint64(nu) + j)
    return _f32(2.0 * u - 1.0)


def model(name: str) -> Model:
    return MODELS[name]()


# --------------------------------------------------------------------------------------
# seeded initial states and actions
# --------------------------------------------------------------------------------------

def initial_state(m: Model, config: int, n_envs: int, env0: int = 0, noise: Optional[float] = None):
    """qpos [N, nq], qvel [N, nv] float32.  Draws 0 .. nq+nv-1 of each env's stream.
    noise=None uses the workload's recipe: cartpole U(+-0.1) on qpos and qvel, the others
    start at rest in the reference configuration."""
    seeds = env_seeds(config, n_envs, env0)[:, None]
    nq, nv = m.nq, m.nv
    q0 = np.zeros(nq) if m.qpos_init is None else m.qpos_init.astype(np.float64)
    if noise is None:
        noise = 0.1 if m.name == "cartpole" else 0.0
    u = uniform01(seeds, np.arange(nq + nv, dtype=np.uint64)[None, :])
    qpos = q0[None, :] + noise * (2.0 * u[:, :nq] - 1.0)
    qvel = noise * (2.0 * u[:, nq:] - 1.0)
    return _f32(qpos), _f32(qvel)


def actions(m: Model, config: int, n_envs: int, t0: int, n_steps: int, env0: int = 0,
            amplitude: float = 0.3) -> np.ndarray:
    """Controls [n_steps, N, nu] float32 for control steps t0 .. t0+n_steps-1.
    Draw index of (t, j) is nq + nv + t*nu + j.  Cartpole: U[-1, 1].  Position-actuated
    models: default_ctrl + U(+-amplitude) when default_ctrl is set, else U(ctrlrange)."""
    seeds = env_seeds(config, n_envs, env0)[None, :, None]
    nu, base = m.nu, m.nq + m.nv
    t = np.arange(t0, t0 + n_steps, dtype=np.uint64)[:, None, None]
    j = np.arange(nu, dtype=np.uint64)[None, None, :]
    u = uniform01(seeds, np.uint64(base) + t * np.uint64(nu) + j)
    if m.default_ctrl is not None:
        out = m.default_ctrl.astype(np.float64)[None, None, :] + amplitude * (2.0 * u - 1.0)
    else:
        lo = m.act_ctrlrange[:, 0].astype(np.float64)
        hi = m.act_ctrlrange[:, 1].astype(np.float64)
        out = lo + (hi - lo) * u
    return _f32(out)
