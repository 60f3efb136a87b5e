"""CPU-only checks of the C ABI library: it loads, exports every function include/pg.h
declares, and the host-side model compiler validates descriptions (no GPU work)."""
import ctypes as C
import dataclasses
import os
import re

import numpy as np
import pytest

from paper_2502_08844_b300 import workloads as W
from tests import models_for_tests as MT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "pg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(pg_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_function():
    from paper_2502_08844_b300 import _capi
    names = header_functions()
    assert len(names) >= 11
    lib = C.CDLL(_capi.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_capi.EXPORTS)


def test_model_compile_sizes():
    from paper_2502_08844_b300 import core
    q = core.CompiledModel(W.quadruped())
    s = q.sizes
    assert (s.nq, s.nv, s.nu, s.nbody, s.nslot) == (19, 18, 12, 10, 4)
    assert s.nrow_max == 4 * 4 + 12
    c = core.CompiledModel(W.cartpole())
    assert (c.sizes.nq, c.sizes.nv, c.sizes.nu, c.sizes.nslot, c.sizes.nrow_max) == (2, 2, 1, 0, 0)


def _broken(mutate):
    m = W.quadruped()
    mutate(m)
    return m


@pytest.mark.parametrize("mutate,code", [
    (lambda m: m.body_parent.__setitem__(2, 5), -1),                     # parent after child
    (lambda m: m.jnt_type.__setitem__(3, 7), -1),                        # bad joint type
    (lambda m: m.jnt_axis.__setitem__(slice(3, 4), 0.0), -1),           # zero hinge axis
    (lambda m: m.pair_geom.__setitem__((0, 0), m.pair_geom[0, 1]) or m.pair_geom.__setitem__((0, 1), 0), -4),  # sphere-plane order
    (lambda m: m.pair_condim.__setitem__(0, 6), -4),                     # condim 6
    (lambda m: setattr(m, "cone", 2), -1),                                # unknown cone
    (lambda m: setattr(m, "cone", W.ELLIPTIC) or setattr(m, "impratio", 2.0), -4),   # elliptic needs impratio 1
    (lambda m: setattr(m, "timestep", 0.0), -1),
    (lambda m: m.act_jnt.__setitem__(0, 0), -1),                         # actuator on the free joint
])
def test_model_compile_rejects_bad_descriptions(mutate, code):
    from paper_2502_08844_b300 import core, _capi
    with pytest.raises(_capi.PgError) as ei:
        core.CompiledModel(_broken(mutate))
    assert ei.value.code == code
    assert len(_capi.pg_last_error()) > 0


def test_null_arguments_are_errors():
    from paper_2502_08844_b300 import _capi
    lib = _capi._lib
    assert lib.pg_model_compile(None, None) == _capi.PG_EINVAL
    assert lib.pg_step(None, None, None, 1, None) == _capi.PG_EINVAL
    assert lib.pg_model_info(None, None) == _capi.PG_EINVAL
    assert lib.pg_batch_compile(None, None, 0, 0, None) == _capi.PG_EINVAL


def test_adjoint_scope_and_parameter_rows():
    """pg_model_info reports the adjoint workspace only for models inside the adjoint's scope:
    contacts between a world plane or heightfield and spheres / capsules / boxes (quadruped,
    cartpole, the rough-terrain quadruped), not the
    hand (box-box, capsule-box) nor the humanoid (capsule-capsule self contact)."""
    from paper_2502_08844_b300 import core
    from tests import models_for_tests as MT
    for m, ok in [(W.quadruped(), True), (W.cartpole(), True), (MT.box_and_capsule_on_plane(), True),
                  (MT.limited_arm(), True), (W.hand(), False), (W.humanoid(), False)]:
        s = core.CompiledModel(m).sizes
        assert (s.adjoint_workspace_bytes > 0) == ok, m.name
        assert s.nparam == m.nbody + m.nv + m.nu
        if ok:
            assert s.adjoint_workspace_bytes >= s.workspace_bytes
    q = W.quadruped()
    q.act_forcelimited = np.ones(q.nu, np.int32)
    q.act_forcerange = np.tile(np.array([[-4.0, 4.0]], np.float32), (q.nu, 1))
    assert core.CompiledModel(q).sizes.adjoint_workspace_bytes > 0       # torque limits: inside
    assert core.CompiledModel(W.quadruped_rough()).sizes.adjoint_workspace_bytes > 0    # heightfield: inside


def test_cylinder_pairs_and_scope():
    """A cylinder pairs with a plane only (4 candidate points) and is inside the adjoint's scope."""
    from paper_2502_08844_b300 import core, _capi
    b = W.ModelBuilder("cyl")
    g0 = b.geom(0, W.PLANE, (0, 0, 0))
    body = b.body(0, (0, 0, 0.2))
    b.joint(body, W.FREE)
    g1 = b.geom(body, W.CYLINDER, (0.05, 0.1), mass=1.0)
    b.pair(g0, g1)
    s = core.CompiledModel(b.build(timestep=0.002)).sizes
    assert s.nslot == 4 and s.nrow_max == 16 and s.adjoint_workspace_bytes > 0
    g2 = b.geom(body, W.SPHERE, (0.05,), mass=0.0)
    b.pair(g0, g2)
    m = b.build(timestep=0.002)
    m.pair_geom[1] = (g2, g1)                    # sphere-cylinder: not a supported pair
    with pytest.raises(_capi.PgError) as ei:
        core.CompiledModel(m)
    assert ei.value.code == _capi.PG_EUNSUPPORTED


def test_friction_loss_rows_and_scope():
    from paper_2502_08844_b300 import core, _capi
    m = W.quadruped()
    m.dof_frictionloss = np.zeros(m.nv, np.float32); m.dof_frictionloss[6:] = 0.5
    s = core.CompiledModel(m).sizes
    assert s.nrow_max == 4 * 4 + 12 + 12 and s.adjoint_workspace_bytes > 0
    h = W.hand(cone=W.ELLIPTIC, frictionloss=0.05)   # friction loss beside the elliptic cone
    hs = core.CompiledModel(h).sizes
    assert hs.nrow_max == core.CompiledModel(W.hand_elliptic()).sizes.nrow_max + 16
    m.dof_frictionloss[7] = -1.0
    with pytest.raises(_capi.PgError) as ei:
        core.CompiledModel(m)
    assert ei.value.code == _capi.PG_EINVAL


def test_per_environment_parameter_rows():
    from paper_2502_08844_b300 import core
    for f in (W.quadruped, W.cartpole, W.humanoid):
        m = f()
        assert core.CompiledModel(m).sizes.nrand == 2 + 4 * m.nbody + 2 * m.nv + 3 * m.nu
    q = W.quadruped()
    q.act_forcelimited = np.ones(q.nu, np.int32)
    q.act_forcerange = np.tile(np.array([[4.0, -4.0]], np.float32), (q.nu, 1))
    from paper_2502_08844_b300 import _capi
    with pytest.raises(_capi.PgError) as ei:
        core.CompiledModel(q)
    assert ei.value.code == _capi.PG_EINVAL


@pytest.mark.parametrize("ndof,ok", [(64, True), (65, False)])
def test_dof_capacity_limit(ndof, ok):
    """The kernels take at most 64 dofs (and 64 bodies, the world included): a floating base
    with 58 hinges (64 dofs, 60 bodies) compiles, one more hinge does not."""
    from paper_2502_08844_b300 import core, _capi
    if ok:
        assert core.CompiledModel(MT.floating_chain(ndof)).sizes.nv == ndof
    else:
        with pytest.raises(_capi.PgError) as ei:
            core.CompiledModel(MT.floating_chain(ndof))
        assert ei.value.code == _capi.PG_ECAPACITY


def test_row_capacity_limit():
    """At most 128 constraint rows: a free body on 33 sphere feet (4 rows per contact) compiles
    with 32 simultaneous contacts (128 rows), not with 33."""
    from paper_2502_08844_b300 import core, _capi
    m33 = MT.many_feet(33)
    with pytest.raises(_capi.PgError) as ei:
        core.CompiledModel(m33)
    assert ei.value.code == _capi.PG_ECAPACITY
    m32 = MT.many_feet(33, max_contacts=32)
    assert core.CompiledModel(m32).sizes.nrow_max == 128


def test_branch_plan_of_the_workload_models():
    """pg_model_branch_plan (host only): the quadruped (4 legs under the torso) and the humanoid
    (2 legs, 2 arms under pelvis and waist) qualify for the branch-parallel kernel with 4 lanes, on
    the plane and on the rough terrain; the cartpole (one chain), the hand (more candidate contact
    points than max_contacts) and the hulls (free bodies, no branch) do not, and the plan says
    why."""
    from paper_2502_08844_b300 import core
    for name in ("quadruped", "humanoid", "quadruped_rough", "humanoid_rough"):
        p = core.CompiledModel(W.model(name)).branch_plan()
        assert p["branch"] and p["lanes_per_env"] == 4 and p["branches"] == 4, (name, p)
    p = core.CompiledModel(W.cartpole()).branch_plan()
    assert not p["branch"] and "fewer than 2 branches" in p["reason"]
    p = core.CompiledModel(W.hand()).branch_plan()
    assert not p["branch"] and "max_contacts" in p["reason"]
    p = core.CompiledModel(W.hulls()).branch_plan()
    assert not p["branch"] and "fewer than 2 branches" in p["reason"]
