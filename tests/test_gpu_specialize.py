"""pg_batch_specialize: the step kernel compiled at run time (NVRTC) with the model as constants
runs the same source as the generic kernel.  With the model known the compiler may fold known
zeros and forward stored constants, which can regroup an FMA, so trajectories agree to rounding
(1e-6 of their scale over a few steps; often bitwise).  Mixed batches keep the generic kernel."""
import numpy as np
import pytest
import torch

from paper_2502_08844_b300 import _capi, core
from paper_2502_08844_b300 import workloads as W
from tests.gpu_helpers import GpuRun

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mname,cfg,n,T", [("quadruped", 1, 300, 6), ("cartpole", 0, 77, 6), ("hand_elliptic", 2, 40, 3),
                                          ("humanoid", 3, 50, 3)])
def test_specialised_kernel_matches_generic(mname, cfg, n, T):
    m = W.model(mname)
    q0, v0 = W.initial_state(m, cfg, n)
    U = W.actions(m, cfg, n, 0, T)
    out = []
    for spec in (False, True):
        run = GpuRun(m, n)
        if spec:
            run.batch.specialize()
        run.set_state(q0, v0)
        tq, tv = run.rollout(U, m.n_substeps, keep=True)
        out.append((tq, tv, run.status()))
    for k in (0, 1):
        a, b = out[0][k], out[1][k]
        assert np.abs(a - b).max() <= 1e-6 * max(np.abs(a).max(), 1.0), (k, np.abs(a - b).max())
    assert np.array_equal(out[0][2], out[1][2])


def test_specialise_keeps_mixed_batches_generic():
    parts = [(core.CompiledModel(W.cartpole()), 4), (core.CompiledModel(W.quadruped()), 4)]
    batch = core.Batch(parts)
    with pytest.raises(_capi.PgError) as ei:
        batch.specialize()
    assert ei.value.code == _capi.PG_EUNSUPPORTED


def test_specialised_adjoint_matches_generic():
    """pg_step_vjp on a specialised batch (specialised forward, tape replay and reverse sweep)
    against the generic kernels: the same rollout gradient up to rounding."""
    import dataclasses
    from tests.test_gpu_adjoint import gpu_rollout_grad
    from oracle import oracle as O
    m = dataclasses.replace(W.quadruped(), iterations=100)
    q0, v0 = W.initial_state(m, 4, 8)
    U = W.actions(m, 4, 8, 0, 8)
    w = O.tracking_loss_weights(O.OracleModel(m))
    a = gpu_rollout_grad(m, q0, v0, U, w)
    b = gpu_rollout_grad(m, q0, v0, U, w, specialize=True)
    for k in ("q0", "v0", "u", "mass", "damping", "kp"):
        x, y = a[k], b[k]
        assert np.abs(x - y).max() <= 1e-4 * max(np.abs(x).max(), 1e-6), (k, np.abs(x - y).max())
