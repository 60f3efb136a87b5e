"""pg_step_vjp_noalloc (the adjoint on a fixed static scratch array) against pg_step_vjp (the
adjoint on library-allocated scratch): two calls in a row, same results.  Called through the C
ABI.  This file is collected last; it must pass alone in a fresh process and after the rest."""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest
import torch

from paper_2502_08844_b300 import _capi, core
from paper_2502_08844_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _setup(n=8, K=3, specialize=False):
    m = dataclasses.replace(W.quadruped(), iterations=100)
    cm = core.CompiledModel(m)
    batch = core.Batch([(cm, n)])
    if specialize:   # True: the branch-parallel tape replay; "thread": the specialised thread kernels
        batch.specialize(branch=specialize is True)
    st = core.State(batch)
    ld = st.ld
    q0, v0 = W.initial_state(m, 4, n)
    st.qpos.copy_(torch.from_numpy(core.to_soa(q0, ld, batch.nq_max)))
    st.qvel.copy_(torch.from_numpy(core.to_soa(v0, ld, batch.nv_max)))
    U = W.actions(m, 4, n, 0, K)
    ctrl = torch.zeros((K, batch.nu_max, ld), device="cuda")
    ctrl[:, :m.nu, :n] = torch.from_numpy(U.transpose(0, 2, 1).copy())
    g = torch.Generator().manual_seed(11)
    gq = torch.randn((K, batch.nq_max, ld), generator=g).cuda()
    gv = torch.randn((K, batch.nv_max, ld), generator=g).cuda()
    aq = torch.randn((batch.nq_max, ld), generator=g).cuda()
    av = torch.randn((batch.nv_max, ld), generator=g).cuda()
    return batch, st, ctrl, gq, gv, aq, av


def _run(entry, batch, st, ctrl, gq, gv, aq, av):
    K, ld = ctrl.shape[0], st.ld
    adj_q, adj_v = aq.clone(), av.clone()
    g_ctrl = torch.zeros_like(ctrl)
    g_par = torch.zeros((batch.nparam_max, ld), device="cuda")
    p = lambda t: torch.cuda.current_stream().cuda_stream if t is None else t.data_ptr()
    entry(batch.handle, st.c(), ctrl.data_ptr(), K, 0, gq.data_ptr(), gv.data_ptr(), adj_q.data_ptr(),
          adj_v.data_ptr(), g_ctrl.data_ptr(), g_par.data_ptr(), p(None))
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in (adj_q, adj_v, g_ctrl, g_par)]


@pytest.mark.parametrize("specialize", [pytest.param(False, id="generic"), pytest.param("thread", id="specialised"),
                                        pytest.param(True, id="branch")])
def test_noalloc_vjp_matches_vjp_on_two_calls_in_a_row(specialize):
    batch, st, ctrl, gq, gv, aq, av = _setup(specialize=specialize)
    q_before = st.qpos.clone()
    ref = _run(_capi.pg_step_vjp, batch, st, ctrl, gq, gv, aq, av)
    first = _run(_capi.pg_step_vjp_noalloc, batch, st, ctrl, gq, gv, aq, av)
    second = _run(_capi.pg_step_vjp_noalloc, batch, st, ctrl, gq, gv, aq, av)
    for a, b, c in zip(ref, first, second):
        assert np.isfinite(a).all()
        assert np.array_equal(a, b)
        assert np.array_equal(a, c)
    assert torch.equal(st.qpos, q_before)   # the checkpoint is read only


def test_noalloc_vjp_leaves_device_memory_unchanged():
    """Free device memory is the same before and after two calls (after one warm-up call, which
    may load the kernels' code), with every buffer allocated beforehand."""
    batch, st, ctrl, gq, gv, aq, av = _setup()
    K, ld = ctrl.shape[0], st.ld
    g_ctrl = torch.zeros_like(ctrl)
    g_par = torch.zeros((batch.nparam_max, ld), device="cuda")
    s = torch.cuda.current_stream().cuda_stream

    def call():
        _capi.pg_step_vjp_noalloc(batch.handle, st.c(), ctrl.data_ptr(), K, 0, gq.data_ptr(), gv.data_ptr(),
                                  aq.data_ptr(), av.data_ptr(), g_ctrl.data_ptr(), g_par.data_ptr(), s)
    call()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    call()
    call()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_vjp_rejects_calls_beyond_its_scratch():
    batch, st, ctrl, gq, gv, aq, av = _setup(n=8, K=1)
    K = 100000   # needs far more than the fixed 16 MiB
    with pytest.raises(_capi.PgError) as ei:
        _capi.pg_step_vjp_noalloc(batch.handle, st.c(), ctrl.data_ptr(), K, 0, None, None, aq.data_ptr(),
                                  av.data_ptr(), ctrl.data_ptr(), aq.data_ptr(), None)
    assert ei.value.code == _capi.PG_ECAPACITY
    assert "16 MiB" in str(ei.value)
