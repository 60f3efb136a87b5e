"""The bench's multi-GPU path is replicas (environments are independent; no data-path
collective).  Its host logic runs here as two gloo ranks on the CPU: disjoint contiguous env
ranges, and the whole-job rate over the slowest rank (MAX all-reduce of the timed seconds)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2502_08844_b300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    n, steps = 64, 10
    secs = [1.5, 2.0][rank]
    rate, worst = bench.whole_job_rate(secs, ws, n, steps, dist)
    m = W.quadruped()
    q, v = W.initial_state(m, 1, n, bench.replica_env0(rank, n))
    out[rank] = (rate, worst, q.tobytes())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_rate_and_env_ranges():
    ws = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        rate, worst, _ = res[r]
        assert worst == 2.0
        assert rate == pytest.approx(ws * 64 * 10 / 2.0)
    # the ranks' inputs are the two halves of one 128-env job
    m = W.quadruped()
    q_all, _ = W.initial_state(m, 1, 128, 0)
    q0 = np.frombuffer(res[0][2], dtype=q_all.dtype).reshape(64, m.nq)
    q1 = np.frombuffer(res[1][2], dtype=q_all.dtype).reshape(64, m.nq)
    assert np.array_equal(q0, q_all[:64]) and np.array_equal(q1, q_all[64:])
