"""Algorithmic FP32 flop count of the physics step (the numerator of the ALU roofline).

The count is the FP64 oracle's own, taken on its counting scalar: every floating-point operation
on a value that depends on the state, the controls or the solver counts one flop (add, sub, mul,
div, sqrt, a transcendental; a fused multiply-add two), operations a model-specialised program
folds count nothing (on constants only, products with a constant 0 or +-1, sums with a constant
0), and the methods counted are the tree methods of the step: CRBA for M and the leaves-first
L^T D L for every factorisation (no fill on a tree pattern).  The solver's contact-force output
is not part of the step.

Per substep the count is fitted, per model, as

    A + B * rows + C * iters + E * rows * iters

with rows the constraint rows assembled and iters the Newton iterations of the substep; the step
kernels' optional solver counters give their sums over a launch, so a launch's count is
A * substeps + B * sum(rows) + C * sum(iters) + E * sum(rows * iters).  The fitted coefficients
are stored in flop_counts.json beside this file; the oracle's own script (oracle/count_flops.py)
writes them and a CPU test refits and checks them.
"""
from __future__ import annotations

import dataclasses
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
COUNTS = os.path.join(HERE, "flop_counts.json")


@dataclasses.dataclass
class FlopModel:
    A: float
    B: float
    C: float
    E: float

    def substeps(self, n_substeps: float, sum_rows: float, sum_iters: float, sum_rows_iters: float) -> float:
        return self.A * n_substeps + self.B * sum_rows + self.C * sum_iters + self.E * sum_rows_iters


def stored_counts() -> dict:
    with open(COUNTS) as f:
        return json.load(f)["models"]


def flop_model(m) -> FlopModel:
    """The counted per-substep flop model of a workload model (by its name)."""
    c = stored_counts()
    if m.name not in c:
        raise KeyError("no counted flops stored for model %r (oracle/count_flops.py --write)" % m.name)
    e = c[m.name]
    return FlopModel(e["A"], e["B"], e["C"], e["E"])


def fp32_peak_tflops(sm_count: int, sm_mhz: float) -> float:
    """CUDA-core FP32 peak: SMs x 128 FP32 lanes x 2 (fma) x clock."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12
