"""The counted flops of the step (the roofline's numerator): the oracle on its counting scalar
(oracle/orc_count.hpp), pinned on textbook kernels with closed-form counts, checked to compute
the oracle's own values, and the stored per-model fit (paper_2502_08844_b300/flop_counts.json,
written by oracle/count_flops.py) reproduced from the oracle."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_08844_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("n", range(1, 10))
def test_counting_scalar_on_textbook_kernels(n):
    """Closed forms: y = A x costs n products and n - 1 sums per row (the first sum is onto the
    constant zero); with A a constant zero matrix nothing; Cholesky column j costs 2j + 1 for the
    pivot (products, sums, sqrt) and 2j + 1 per row below (products, sums, division), its two
    triangular solves 2i + 1 per row each; the leaves-first L^T D L of an arrowhead (a root dof
    coupled to n - 1 leaves) makes no fill: 3 flops per leaf, and its solve 2 + 2 per leaf plus one
    division per dof.  A count that takes copies, constant zeros or fill as work fails one of these."""
    assert O.count_selftest(0, n) == 2 * n * n - n
    assert O.count_selftest(1, n) == 0
    chol = sum((2 * j + 1) * (n - j) for j in range(n)) + 2 * n * n
    assert O.count_selftest(2, n) == chol
    assert O.count_selftest(3, n) == 8 * n - 7


@pytest.mark.parametrize("name,cfg", [("quadruped", 1), ("humanoid", 3), ("hand", 2), ("cartpole", 0)])
def test_crba_equals_the_kinetic_energy_mass_matrix(name, cfg):
    """The counted instantiation takes CRBA for M; it must be the oracle's kinetic-energy M."""
    m = W.model(name)
    om = O.OracleModel(m)
    q, _ = W.initial_state(m, cfg, 4, noise=0.3)
    for e in range(4):
        A, B = om.mass_matrix(q[e]), om.mass_matrix_crba(q[e])
        assert np.abs(A - B).max() <= 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("name,cfg", [("quadruped", 1), ("humanoid", 3), ("hand", 2)])
def test_counted_oracle_computes_the_oracle_step(name, cfg):
    """The counting scalar carries the oracle's doubles; only the factorisations (L^T D L instead of
    Cholesky) and M (CRBA) differ, which moves the result by rounding only."""
    m = W.model(name)
    om = O.OracleModel(m)
    q0, v0 = W.initial_state(m, cfg, 2)
    U = W.actions(m, cfg, 2, 0, 2)
    for e in range(2):
        q, v, w = q0[e].astype(float), v0[e].astype(float), np.zeros(m.nv)
        for t in range(2):
            _, rows, iters, q, v, w = O.count_substeps(om, q, v, w, U[t, e], m.n_substeps)
        qo, vo, _, _ = om.rollout(q0[e:e + 1], v0[e:e + 1], U[:, e:e + 1], m.n_substeps)
        assert np.abs(q - qo[0]).max() <= 1e-9 * max(1.0, np.abs(qo).max())
        assert np.abs(v - vo[0]).max() <= 1e-9 * max(1.0, np.abs(vo).max())


def test_stored_flop_fit_is_the_oracles():
    """paper_2502_08844_b300/flop_counts.json (the bench's roofline numerator) equals a fresh fit of
    the counted oracle, and the fit explains the sampled substeps."""
    from oracle import count_flops
    stored = json.load(open(os.path.join(ROOT, "paper_2502_08844_b300", "flop_counts.json")))["models"]
    fresh = count_flops.run()
    assert set(stored) == set(fresh)
    for name, f in fresh.items():
        for k in ("A", "B", "C", "E"):
            assert abs(stored[name][k] - f[k]) <= 1e-6 * max(1.0, abs(f[k])), (name, k)
        assert f["mean_rel_residual"] <= 0.1, (name, f["mean_rel_residual"])
