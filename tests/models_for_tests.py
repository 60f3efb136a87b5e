"""Small hand-built models used only by the tests (inputs; no physics arithmetic)."""
from __future__ import annotations

import math

from paper_2502_08844_b300 import workloads as W


def planar_chain(n_links=3, length=0.5, mass=1.0, radius=0.02, gravity=(0, 0, -9.81), damping=0.0,
                 timestep=0.001, limited=False):
    """n hinge links about y, each a capsule of `length` hanging along -z from its hinge."""
    b = W.ModelBuilder("chain%d" % n_links)
    parent, pos = 0, (0, 0, 0)
    for i in range(n_links):
        body = b.body(parent, pos)
        b.joint(body, W.HINGE, axis=(0, 1, 0), damping=damping, limited=limited, range=(-1.0, 1.0))
        b.geom(body, W.CAPSULE, (radius, length / 2), pos=(0, 0, -length / 2), mass=mass)
        parent, pos = body, (0, 0, -length)
    return b.build(timestep=timestep, gravity=gravity)


def free_body(gravity=(0, 0, -9.81), timestep=0.01, inertia=None, mass=2.0, z0=1.0, geom=True):
    """One free body; with inertia=(xx,yy,zz,xy,xz,yz) the mass properties are explicit (COM at the origin)."""
    b = W.ModelBuilder("free_body")
    if inertia is None:
        body = b.body(0, (0, 0, z0))
        b.geom(body, W.BOX, (0.1, 0.2, 0.3), mass=mass)
    else:
        body = b.body(0, (0, 0, z0), mass=mass, inertia=inertia, geom_inertia=False)
    b.joint(body, W.FREE)
    return b.build(timestep=timestep, gravity=gravity)


def sphere_on_plane(mass=1.0, radius=0.1, friction=0.0, condim=1, timestep=0.002, z0=None, iterations=50):
    b = W.ModelBuilder("sphere_on_plane")
    floor = b.geom(0, W.PLANE, (0, 0, 0))
    body = b.body(0, (0, 0, radius if z0 is None else z0))
    b.joint(body, W.FREE)
    s = b.geom(body, W.SPHERE, (radius,), mass=mass)
    b.pair(floor, s, friction=friction, condim=condim)
    return b.build(timestep=timestep, iterations=iterations)


def pendulum(length=1.0, mass=1.0, radius=0.02, timestep=0.001):
    """A single capsule on a hinge about y (compound pendulum)."""
    b = W.ModelBuilder("pendulum")
    body = b.body(0, (0, 0, 0))
    b.joint(body, W.HINGE, axis=(0, 1, 0))
    b.geom(body, W.CAPSULE, (radius, length / 2), pos=(0, 0, -length / 2), mass=mass)
    return b.build(timestep=timestep)


def quadruped_zero_gravity(timestep=0.004):
    m = W.quadruped()
    m.gravity[:] = 0.0
    m.pair_geom = m.pair_geom[:0]
    m.pair_friction = m.pair_friction[:0]
    m.pair_condim = m.pair_condim[:0]
    m.jnt_limited[:] = 0
    m.timestep = timestep
    m.max_contacts = 0
    return m


def arm_with_slider(gravity=(0, 0, 0), timestep=0.001):
    """Hinge (y) arm carrying a slider along the arm's x axis and a second hinge at the slider:
    exercises slide joints on rotating frames."""
    b = W.ModelBuilder("arm_slider")
    arm = b.body(0, (0, 0, 0))
    b.joint(arm, W.HINGE, axis=(0, 1, 0))
    b.geom(arm, W.CAPSULE, (0.02, 0.2), pos=(0.2, 0, 0), quat=(0.7071068, 0, 0.7071068, 0), mass=0.5)
    slider = b.body(arm, (0.1, 0, 0))
    b.joint(slider, W.SLIDE, axis=(1, 0, 0))
    b.geom(slider, W.BOX, (0.05, 0.04, 0.03), pos=(0.02, 0.01, 0.0), mass=0.8)
    tip = b.body(slider, (0.05, 0, 0.02))
    b.joint(tip, W.HINGE, axis=(0, 0.6, 0.8))
    b.geom(tip, W.CAPSULE, (0.02, 0.1), pos=(0, 0, -0.1), mass=0.3)
    return b.build(timestep=timestep, gravity=gravity)


def quadruped_passive(timestep=0.004, gravity=(0, 0, 0)):
    """The quadruped without actuation, limits or contacts (a free-floating passive tree)."""
    m = quadruped_zero_gravity(timestep)
    m.gravity[:] = gravity
    m.act_kp[:] = 0.0
    m.act_kd[:] = 0.0
    return m


def box_and_capsule_on_plane(timestep=0.002, iterations=100, friction=1.0):
    """A tilted free box and a tilted free capsule resting on the floor plane: box-corner and
    capsule-end contacts (pyramidal), for the adjoint's plane-contact features."""
    b = W.ModelBuilder("box_capsule_plane")
    floor = b.geom(0, W.PLANE, (0, 0, 0))
    box = b.body(0, (0, 0, 0.2))
    b.joint(box, W.FREE)
    g1 = b.geom(box, W.BOX, (0.05, 0.04, 0.03), mass=0.8)
    cap = b.body(0, (0.5, 0, 0.2))
    b.joint(cap, W.FREE)
    g2 = b.geom(cap, W.CAPSULE, (0.02, 0.08), mass=0.3)
    b.pair(floor, g1, friction=friction, condim=3)
    b.pair(floor, g2, friction=friction, condim=3)
    return b.build(timestep=timestep, iterations=iterations, n_substeps=4)


def limited_arm(timestep=0.002, iterations=100):
    """Two-link arm under gravity with PD actuators driving both hinges into their limits."""
    b = W.ModelBuilder("limited_arm")
    l1 = b.body(0, (0, 0, 0))
    j1 = b.joint(l1, W.HINGE, axis=(0, 1, 0), limited=True, range=(-0.4, 0.5), damping=0.05)
    b.geom(l1, W.CAPSULE, (0.03, 0.15), pos=(0, 0, -0.15), mass=0.6)
    l2 = b.body(l1, (0, 0, -0.3))
    j2 = b.joint(l2, W.HINGE, axis=(0.3, 0.9, 0.3), limited=True, range=(-0.6, 0.3), damping=0.02)
    b.geom(l2, W.CAPSULE, (0.02, 0.1), pos=(0, 0, -0.1), mass=0.3)
    b.actuator(j1, W.POSITION, kp=8.0, kd=0.2)
    b.actuator(j2, W.POSITION, kp=3.0, kd=0.1)
    return b.build(timestep=timestep, iterations=iterations, n_substeps=4)


def floating_chain(ndof):
    """A floating base (6 dofs) carrying a chain of ndof - 6 hinged links (alternating x and y
    axes), with joint damping: 64 dofs is the kernels' limit."""
    b = W.ModelBuilder("chain%d" % ndof)
    base = b.body(0, (0.0, 0.0, 2.0))
    b.joint(base, W.FREE)
    b.geom(base, W.BOX, (0.05, 0.05, 0.05), mass=1.0)
    parent = base
    for i in range(ndof - 6):
        body = b.body(parent, (0.0, 0.0, -0.05))
        b.joint(body, W.HINGE, axis=(0, 1, 0) if i % 2 else (1, 0, 0), damping=0.01)
        b.geom(body, W.CAPSULE, (0.01, 0.02), pos=(0, 0, -0.025), mass=0.05)
        parent = body
    return b.build(timestep=0.002, iterations=4)


def many_feet(nfeet, max_contacts=None):
    """A free plate on nfeet sphere feet over a plane, each foot a contact pair (4 pyramid rows
    per contact: 32 simultaneous contacts is the kernels' 128-row limit)."""
    b = W.ModelBuilder("feet%d" % nfeet)
    floor = b.geom(0, W.PLANE, (0, 0, 0))
    body = b.body(0, (0, 0, 0.0795))
    b.joint(body, W.FREE)
    b.geom(body, W.BOX, (1.0, 1.0, 0.05), mass=1.0)
    for k in range(nfeet):
        g = b.geom(body, W.SPHERE, (0.02,), pos=(-0.9 + 0.05 * k, 0.02 * (k % 3), -0.06))
        b.pair(floor, g, friction=1.0, condim=3)
    return b.build(timestep=0.002, iterations=6, max_contacts=max_contacts, qpos_init=(0, 0, 0.0795, 1, 0, 0, 0))


def floating_star(ndof):
    """A floating plate (6 dofs) with ndof - 6 single hinged legs around its rim, alternating
    radial and tangential axes: the 64-dof limit on a shallow, well-conditioned tree."""
    b = W.ModelBuilder("star%d" % ndof)
    base = b.body(0, (0.0, 0.0, 2.0))
    b.joint(base, W.FREE)
    b.geom(base, W.BOX, (0.2, 0.2, 0.05), mass=2.0)
    for i in range(ndof - 6):
        ang = 2 * math.pi * i / (ndof - 6)
        c, s = math.cos(ang), math.sin(ang)
        body = b.body(base, (0.15 * c, 0.15 * s, 0.0))
        b.joint(body, W.HINGE, axis=(c, s, 0) if i % 2 else (-s, c, 0), damping=0.01)
        b.geom(body, W.CAPSULE, (0.01, 0.05), pos=(0, 0, -0.05), mass=0.1)
    return b.build(timestep=0.002, iterations=4)
