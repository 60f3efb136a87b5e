"""The linear algebra the branch-parallel kernel relies on, checked in FP64 on the oracle's own
matrices (no GPU): with the dofs ordered branch by branch and the trunk last, the mass matrix M
and the Newton Hessian H = M + J^T D J are block arrowheads; a solve through the branch blocks and
the trunk's Schur complement equals the dense solve; and each row's
A_hat = (J M^-1 J^T)_rr equals z^T z + |L_S^-1 (v - Y^T z)|^2 with z = L_B^-1 u, for the row's
branch part u and trunk part v (the oracle's A_hat is the dense definition, reading R11).

Branches follow the branch plan's rule: from each leaf body, climb through bodies without a free
joint while the parent has that one child; stop below the world, a free body or a body with
several children.  Everything else is trunk."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_08844_b300 import core
from paper_2502_08844_b300 import workloads as W


def _dofs_of_bodies(m):
    """dof indices of each body (joints in order; a free joint has 6 dofs)."""
    out = {b: [] for b in range(m.nbody)}
    d = 0
    for j in range(m.njnt):
        k = 6 if m.jnt_type[j] == W.FREE else 1
        out[int(m.jnt_body[j])] += list(range(d, d + k))
        d += k
    return out


def _branches(m):
    parent = [int(p) for p in m.body_parent]
    children = {b: [c for c in range(m.nbody) if parent[c] == b] for b in range(m.nbody)}
    free = {int(m.jnt_body[j]) for j in range(m.njnt) if m.jnt_type[j] == W.FREE}
    out = []
    for leaf in range(1, m.nbody):
        if children[leaf] or leaf in free:
            continue
        chain, b = [leaf], leaf
        while True:
            p = parent[b]
            if p <= 0 or p in free or len(children[p]) != 1:
                break
            chain.append(p)
            b = p
        out.append(sorted(chain))
    return out


def _contact_state(m, cfg, t):
    om = O.OracleModel(m)
    q0, v0 = W.initial_state(m, cfg, 2)
    U = W.actions(m, cfg, 2, 0, t + 2)
    _, _, _, _, tq, tv = om.rollout(q0, v0, U, m.n_substeps, trajectory=True)
    return om, om.forward(tq[t, 0], tv[t, 0], ctrl=U[t + 1, 0])


@pytest.mark.parametrize("name,cfg,t,nbranch,ntrunk", [("quadruped", 1, 20, 4, 6), ("humanoid", 3, 10, 4, 9)])
def test_block_arrowhead_solves_and_a_hat(name, cfg, t, nbranch, ntrunk):
    m = W.model(name)
    plan = core.CompiledModel(m).branch_plan()
    branches = _branches(m)
    assert plan["branch"] and plan["branches"] == len(branches) == nbranch
    dofs = _dofs_of_bodies(m)
    bdofs = [sorted(d for b in br for d in dofs[b]) for br in branches]
    in_branch = sorted(d for bd in bdofs for d in bd)
    trunk = [d for d in range(m.nv) if d not in in_branch]
    assert len(trunk) == ntrunk

    om, o = _contact_state(m, cfg, t)
    M, rows = o["M"], o["rows"]
    assert o["nrow"] > 0
    J, D, a_hat = rows[:, :m.nv], rows[:, m.nv + 3], rows[:, m.nv + 4]
    # every row touches at most one branch (and the trunk); the feet's rows touch their leg
    touched = [sum(np.any(J[r, bd] != 0) for bd in bdofs) for r in range(J.shape[0])]
    assert max(touched) == 1
    H = M + (J.T * D) @ J
    for A in (M, H):
        for a in range(nbranch):
            for b in range(nbranch):
                if a != b:
                    assert not np.any(A[np.ix_(bdofs[a], bdofs[b])])   # exactly zero: arrowhead

    rng = np.random.default_rng(0)
    for A in (M, H):
        rhs = rng.standard_normal(m.nv)
        Ls, Ys, zs = [], [], []
        S = A[np.ix_(trunk, trunk)].copy()
        c = rhs[trunk].copy()
        for bd in bdofs:
            L = np.linalg.cholesky(A[np.ix_(bd, bd)])
            Y = np.linalg.solve(L, A[np.ix_(bd, trunk)])
            z = np.linalg.solve(L, rhs[bd])
            S -= Y.T @ Y
            c -= Y.T @ z
            Ls.append(L); Ys.append(Y); zs.append(z)
        x = np.zeros(m.nv)
        x[trunk] = np.linalg.solve(S, c)
        for bd, L, Y, z in zip(bdofs, Ls, Ys, zs):
            x[bd] = np.linalg.solve(L.T, z - Y @ x[trunk])
        ref = np.linalg.solve(A, rhs)
        assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()

    # A_hat of every row from the blocks of M, against the dense J M^-1 J^T and the oracle's column
    Ls = [np.linalg.cholesky(M[np.ix_(bd, bd)]) for bd in bdofs]
    Ys = [np.linalg.solve(L, M[np.ix_(bd, trunk)]) for bd, L in zip(bdofs, Ls)]
    S = M[np.ix_(trunk, trunk)] - sum(Y.T @ Y for Y in Ys)
    LS = np.linalg.cholesky(S)
    dense = np.einsum("ri,ri->r", J, np.linalg.solve(M, J.T).T)
    for r in range(J.shape[0]):
        zz, w = 0.0, J[r, trunk].copy()
        for bd, L, Y in zip(bdofs, Ls, Ys):
            z = np.linalg.solve(L, J[r, bd])
            zz += z @ z
            w -= Y.T @ z
        s = np.linalg.solve(LS, w)
        assert abs(zz + s @ s - dense[r]) <= 1e-10 * dense[r]
        assert abs(a_hat[r] - dense[r]) <= 1e-10 * dense[r]
