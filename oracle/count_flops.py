"""Counted flops of the step -- TEST INFRASTRUCTURE (calls only the oracle and the seeded input
generators).

Runs each workload model through the oracle instantiated on its counting scalar (orc_count.hpp:
every floating-point operation on state-dependent values counts one flop, operations a
model-specialised program folds count nothing, the factorisations are the tree methods) and fits,
per model, the per-substep count

    flops = A + B * rows + C * iters + E * rows * iters

(rows: constraint rows assembled in the substep, iters: its Newton iterations; the step kernels
count both) by least squares over the sampled substeps.  The contact-force output of the solver is
not part of the step and is left out.

    python -m oracle.count_flops            # print the fit
    python -m oracle.count_flops --write    # store it in paper_2502_08844_b300/flop_counts.json

The stored fit is the roofline numerator's model (paper_2502_08844_b300/flops.py);
tests/test_oracle_flops.py refits it from the oracle and checks the stored values.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2502_08844_b300 import workloads as W  # noqa: E402

OUT = os.path.join(ROOT, "paper_2502_08844_b300", "flop_counts.json")
# (model, input config, environments, control steps) sampled per model
SAMPLES = [("cartpole", 0, 4, 10), ("quadruped", 1, 8, 40), ("hand", 2, 4, 20), ("hand_elliptic", 2, 4, 20),
           ("humanoid", 3, 4, 30)]
STEP_PHASES = 8   # kinematics .. integrate; phase 8 (the force output) is not part of the step


def sample(name: str, cfg: int, n_env: int, n_steps: int):
    """(flops, rows, iters) of every substep of n_env environments over n_steps control steps"""
    m = W.model(name)
    om = O.OracleModel(m)
    q0, v0 = W.initial_state(m, cfg, n_env)
    U = W.actions(m, cfg, n_env, 0, n_steps)
    fl, rows, iters, phases = [], [], [], []
    for e in range(n_env):
        q, v, w = q0[e].astype(np.float64), v0[e].astype(np.float64), np.zeros(m.nv)
        for t in range(n_steps):
            c, r, it, q, v, w = O.count_substeps(om, q, v, w, U[t, e], m.n_substeps)
            per_phase = c.sum(axis=2)[:, :STEP_PHASES]
            fl.append(per_phase.sum(axis=1))
            phases.append(per_phase)
            rows.append(r)
            iters.append(it)
    return np.concatenate(fl), np.concatenate(rows), np.concatenate(iters), np.concatenate(phases)


def fit(flops: np.ndarray, rows: np.ndarray, iters: np.ndarray):
    X = np.stack([np.ones_like(flops), rows, iters, rows * iters], axis=1).astype(np.float64)
    coef, *_ = np.linalg.lstsq(X, flops, rcond=None)
    pred = X @ coef
    return coef, pred


def run():
    out = {}
    for name, cfg, n_env, n_steps in SAMPLES:
        fl, rows, iters, phases = sample(name, cfg, n_env, n_steps)
        coef, pred = fit(fl, rows, iters)
        rel = np.abs(pred - fl) / fl
        out[name] = {"A": float(coef[0]), "B": float(coef[1]), "C": float(coef[2]), "E": float(coef[3]),
                     "substeps": int(fl.size), "mean_flops": float(fl.mean()),
                     "max_rel_residual": float(rel.max()), "mean_rel_residual": float(rel.mean()),
                     "mean_phase_flops": {p: float(x) for p, x in zip(O.COUNT_PHASES, phases.mean(axis=0))},
                     "sample": "%d environments x %d control steps of the %s workload (input config %d)"
                               % (n_env, n_steps, name, cfg)}
    return out


if __name__ == "__main__":
    res = run()
    print(json.dumps(res, indent=1))
    if "--write" in sys.argv:
        doc = {"what": "per-substep counted flops of the step, A + B rows + C iters + E rows iters, fitted "
                       "to the oracle on its counting scalar (oracle/count_flops.py)",
               "models": res}
        with open(OUT, "w") as f:
            json.dump(doc, f, indent=1)
            f.write("\n")
        print("wrote", OUT)
