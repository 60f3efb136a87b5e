"""pg_step_ex: the step's optional outputs.  The last substep's contact force of every candidate
slot, in its contact's frame (normal, t1, t2), against the oracle's converged forces of the same
substep (both solvers run to their exact termination), component by component; the active-contact
count; and that asking for the outputs changes nothing in the state."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_08844_b300 import core
from paper_2502_08844_b300 import workloads as W
from tests.gpu_helpers import GpuRun
from tests.test_gpu_parity import box_box_slot_perm

pytestmark = pytest.mark.gpu

FORCE_RTOL = 1e-3


def oracle_slot_forces(m, o):
    """per candidate slot: (f_n, f_t1, f_t2) from the oracle's rows (active slots in order; a pyramid's
    4 edge rows, an elliptic contact's 3 rows (n, t1, t2), a condim-1 contact's 1 row)"""
    nv = m.nv
    f = o["rows"][:, nv + 6]
    out = np.zeros((o["contacts"].shape[0], 3))
    r = 0
    slot_pair = np.repeat(np.arange(m.npair), [_nslot(m, p) for p in range(m.npair)])
    for s in range(out.shape[0]):
        if o["contacts"][s, 0] <= 0:
            continue
        p = slot_pair[s]
        mu = m.pair_friction[p]
        if m.pair_condim[p] == 1:
            out[s] = [f[r], 0, 0]; r += 1
        elif m.cone == W.ELLIPTIC:
            out[s] = f[r:r + 3]; r += 3
        else:
            e = f[r:r + 4]
            out[s] = [e.sum(), mu * (e[0] - e[1]), mu * (e[2] - e[3])]; r += 4
    return out


_SLOTS = {(W.PLANE, W.SPHERE): 1, (W.PLANE, W.CAPSULE): 2, (W.PLANE, W.BOX): 4, (W.SPHERE, W.SPHERE): 1,
          (W.SPHERE, W.CAPSULE): 1, (W.CAPSULE, W.CAPSULE): 1, (W.SPHERE, W.BOX): 1, (W.CAPSULE, W.BOX): 2,
          (W.BOX, W.BOX): 4, (W.PLANE, W.CYLINDER): 4}


def _nslot(m, p):
    return _SLOTS[(int(m.geom_type[m.pair_geom[p, 0]]), int(m.geom_type[m.pair_geom[p, 1]]))]


def _states(m, cfg, times, n_env=3):
    om = O.OracleModel(m)
    q0, v0 = W.initial_state(m, cfg, n_env)
    U = W.actions(m, cfg, n_env, 0, max(times) + 2)
    _, _, _, _, tq, tv = om.rollout(q0, v0, U, m.n_substeps, trajectory=True, nthreads=4)
    return om, [(tq[t, e].astype(np.float32).astype(np.float64), tv[t, e].astype(np.float32).astype(np.float64),
                 U[t + 1, e].astype(np.float64)) for t in times for e in range(n_env)]


@pytest.mark.parametrize("mname,cfg,specialize", [("quadruped", 1, False), ("quadruped", 1, True),
                                                  ("quadruped", 1, "branch"), ("humanoid", 3, "branch"),
                                                  ("hand", 2, True), ("hand_elliptic", 2, False)])
def test_contact_forces_match_converged_oracle(mname, cfg, specialize):
    m = W.model(mname)
    om, states = _states(m, cfg, (0, 4, 19))
    mc = dataclasses.replace(W.model(mname), iterations=100)   # the GPU Newton to its exact termination
    checked = 0
    for q, v, u in states:
        n = 4
        run = GpuRun(mc, n, specialize=specialize)
        run.set_state(np.repeat(q[None], n, 0), np.repeat(v[None], n, 0))
        nslot = core._capi.pg_batch_nslot(run.batch.handle)
        F = torch.zeros((nslot, 3, run.state.ld), device="cuda")
        nc = torch.zeros(run.state.ld, dtype=torch.int32, device="cuda")
        core.step_ex(run.batch, run.state, run.ctrl_tensor(np.repeat(u[None], n, 0)), 1, F, nc)
        torch.cuda.synchronize()
        o = om.forward(q, v, np.zeros(m.nv), u, solver_cap=-1)
        ref = oracle_slot_forces(m, o)
        got = F[:, :, 2].cpu().numpy()
        # a box-box manifold's points in the oracle's slot order, from the GPU's own contacts of
        # the same state (the debug substep)
        dbg = GpuRun(mc, n)
        dbg.set_state(np.repeat(q[None], n, 0), np.repeat(v[None], n, 0))
        gc = dbg.debug(np.repeat(u[None], n, 0), 2)["contacts"]
        got = got[box_box_slot_perm(m, gc, o["contacts"])]
        act = o["contacts"][:, 0] > 0
        assert int(nc[2].item()) == int(act.sum())
        if not act.any():
            continue
        for s in np.where(act)[0]:
            tol = FORCE_RTOL * abs(ref[s, 0]) + 1e-6
            assert np.abs(got[s] - ref[s]).max() <= tol, (s, got[s], ref[s])
        assert np.all(got[~act] == 0)
        checked += 1
    assert checked >= 3


@pytest.mark.parametrize("specialize", [False, True, "branch"])
def test_outputs_change_nothing_in_the_state(specialize):
    m = W.quadruped()
    n = 37
    q0, v0 = W.initial_state(m, 1, n)
    U = W.actions(m, 1, n, 0, 3)
    out = []
    for with_out in (False, True):
        run = GpuRun(m, n, specialize=specialize)
        run.set_state(q0, v0)
        F = torch.zeros((4, 3, run.state.ld), device="cuda")
        for t in range(3):
            if with_out:
                core.step_ex(run.batch, run.state, run.ctrl_tensor(U[t]), 5, F, None)
            else:
                core.step(run.batch, run.state, run.ctrl_tensor(U[t]), 5)
        out.append(run.get())
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_mixed_batch_branch_parts_write_forces_per_model():
    """A mixed batch whose quadruped and humanoid parts run the branch-parallel kernel: the rows of a
    model with fewer slots than the batch's largest are zero; the active counts match the oracle."""
    from tests.gpu_helpers import MixedRun
    parts = [("cartpole", 0, 5), ("quadruped", 1, 6), ("humanoid", 3, 7)]
    run = MixedRun([(W.model(nm), n) for nm, _, n in parts], specialize="branch")
    inits = [W.initial_state(W.model(nm), cfg, n) for nm, cfg, n in parts]
    run.set_state([q for q, _ in inits], [v for _, v in inits])
    us = [W.actions(W.model(nm), cfg, n, 0, 1)[0] for nm, cfg, n in parts]
    nslot = core._capi.pg_batch_nslot(run.batch.handle)
    F = torch.full((nslot, 3, run.state.ld), 7.0, device="cuda")
    nc = torch.zeros(run.state.ld, dtype=torch.int32, device="cuda")
    core.step_ex(run.batch, run.state, run.ctrl_tensor(us), 1, F, nc)
    torch.cuda.synchronize()
    Fh, nch = F.cpu().numpy(), nc.cpu().numpy()
    o = 0
    for (nm, cfg, n), (q0, v0), u in zip(parts, inits, us):
        m = W.model(nm)
        om = O.OracleModel(m)
        for e in range(n):
            r = om.forward(q0[e], v0[e], np.zeros(m.nv), u[e])
            assert nch[o + e] == int((r["contacts"][:, 0] > 0).sum()) if m.npair else nch[o + e] == 0
            assert np.all(Fh[m.npair and sum(_nslot(m, p) for p in range(m.npair)):, :, o + e] == 0)
        o += n
