"""Algorithmic FP32 flop count of the physics step (for the ALU roofline).

Counts what the method needs on the tree-sparse pattern, independent of how the kernel
schedules it: add = mul = 1, fma = 2, div = sqrt = rsqrt = 1, a sin/cos pair = 2.  Per
substep the count is

    A + B * nrow + C * iters + E * nrow * iters

with nrow the constraint rows assembled and iters the Newton iterations of that substep
(the kernel's optional solver counters give their sums).  A covers kinematics, CRBA, the
LDL^T factor, RNEA, the smooth solve, collision and integration; B the per-row Jacobian,
Ahat and reference acceleration; C the per-iteration dense work on nv (Cholesky, solves,
M products); E the per-iteration per-row work (residual, gradient, Hessian update,
line search, active-set check).  Dense Cholesky of H is counted at nv^3/3 because H is
dense in general; everything on M uses the ancestor pattern only.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import workloads as W

_PAIR_COST = {(W.PLANE, W.SPHERE): 25, (W.PLANE, W.CAPSULE): 55, (W.PLANE, W.BOX): 150, (W.SPHERE, W.SPHERE): 30,
              (W.SPHERE, W.CAPSULE): 45, (W.CAPSULE, W.CAPSULE): 70, (W.SPHERE, W.BOX): 60, (W.CAPSULE, W.BOX): 120,
              (W.BOX, W.BOX): 600, (W.PLANE, W.CYLINDER): 80}
_PAIR_SLOTS = {(W.PLANE, W.SPHERE): 1, (W.PLANE, W.CAPSULE): 2, (W.PLANE, W.BOX): 4, (W.SPHERE, W.SPHERE): 1,
               (W.SPHERE, W.CAPSULE): 1, (W.CAPSULE, W.CAPSULE): 1, (W.SPHERE, W.BOX): 1, (W.CAPSULE, W.BOX): 2,
               (W.BOX, W.BOX): 4, (W.PLANE, W.CYLINDER): 4}


@dataclasses.dataclass
class FlopModel:
    A: float
    B: float
    C: float
    E: float

    def substeps(self, n_substeps: float, sum_rows: float, sum_iters: float, sum_rows_iters: float) -> float:
        return self.A * n_substeps + self.B * sum_rows + self.C * sum_iters + self.E * sum_rows_iters


def _dof_tree(m: W.Model):
    nv = m.nv
    dof_body = np.zeros(nv, int)
    parent = -np.ones(nv, int)
    last = {0: -1}
    adr = m.jnt_dofadr()
    for b in range(1, m.nbody):
        prev = last[int(m.body_parent[b])]
        for j in np.where(m.jnt_body == b)[0]:
            for k in range(6 if m.jnt_type[j] == W.FREE else 1):
                d = adr[j] + k
                dof_body[d] = b
                parent[d] = prev
                prev = d
        last[b] = prev
    depth = np.zeros(nv, int)
    for d in range(nv):
        depth[d] = 0 if parent[d] < 0 else depth[parent[d]] + 1
    chain = {0: set()}
    for b in range(1, m.nbody):
        chain[b] = set(chain[int(m.body_parent[b])]) | set(np.where(dof_body == b)[0].tolist())
    return depth, chain


def flop_model(m: W.Model) -> FlopModel:
    nv, nq = m.nv, m.nq
    nb = m.nbody - 1
    depth, chain = _dof_tree(m)
    nnzM = int(np.sum(depth + 1))
    jt = list(m.jnt_type)
    n_hinge, n_slide, n_free = jt.count(W.HINGE), jt.count(W.SLIDE), jt.count(W.FREE)
    # kinematics and derived quantities
    fk = 98 * nb + 129 * n_hinge + 69 * n_slide + 12 * n_free
    derived = 116 * nb + 98 * m.ngeom + 12 * nv
    n_children = sum(1 for b in range(1, m.nbody) if m.body_parent[b] > 0)
    crba = 10 * n_children + 45 * nv + 11 * nnzM
    ldl = int(sum(d + d * (d + 1) for d in depth))
    rnea = 48 * nv + 135 * nb + 11 * nv
    smooth = 2 * nv + 5 * m.nu + 2 * nv + 4 * int(np.sum(depth)) + nv
    coll = 0
    slots = 0
    for p in range(m.npair):
        key = (int(m.geom_type[m.pair_geom[p, 0]]), int(m.geom_type[m.pair_geom[p, 1]]))
        coll += _PAIR_COST[key]
        slots += _PAIR_SLOTS[key]
    coll += 25 * slots
    integ = 2 * nv + sum(1 for t in jt if t != W.FREE) * 2 + n_free * 46
    warm_cost = 2 * (4 * nnzM + 2 * nv)
    A = fk + derived + crba + ldl + rnea + smooth + coll + integ + warm_cost
    # per row: Jacobian share (38 per chain dof per contact, 4 rows), velocity, Ahat, aref, D
    if m.npair:
        nnz = np.mean([len(chain[int(m.geom_body[m.pair_geom[p, 0]])] | chain[int(m.geom_body[m.pair_geom[p, 1]])])
                       for p in range(m.npair)])
        chain_depth = np.mean([np.sum(depth[list(chain[int(m.geom_body[m.pair_geom[p, 1]])])])
                               for p in range(m.npair)])
    else:
        nnz, chain_depth = 1.0, 0.0
    B = 38 * nnz / 4 + 2 * nnz + (2 * chain_depth + 2 * nnz + nv) + 15 + 4 + 3 + 2 * (2 * nnz + 4)
    C = (4 * nnzM + nv) + (nv ** 3 / 3 + nv ** 2 / 2 + nv) + 2 * nv * nv + 4 * nnzM + 4 * nv + 2 * nv
    E = (2 * nnz + 1) + (2 * nnz + 1) + nnz * (nnz + 1) + 2 * nnz + 8 + (2 * nnz + 1)
    return FlopModel(float(A), float(B), float(C), float(E))


def fp32_peak_tflops(sm_count: int, sm_mhz: float) -> float:
    """CUDA-core FP32 peak: SMs x 128 FP32 lanes x 2 (fma) x clock."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12
