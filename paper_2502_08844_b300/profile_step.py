"""Per-launch record of the physics step, for running under a profiler.

Steps one workload model's batch for `--warmup` control steps and then `--steps` more, one launch
each, and prints one JSON line per launch after the warm-up, with that launch's solver counters
(constraint rows, Newton iterations, their product, summed over environments and substeps) and
the algorithmic FP32 flops they give (flops.py, the oracle's counted model).  A profiler that
captures launch number `warmup + k` of the step kernel (`-k regex:pg_step -s <warmup + k> -c 1`)
then has the counted flops of exactly that launch to set its executed instruction counts against.

    python -m paper_2502_08844_b300.profile_step --workload quadruped --envs 256 --warmup 3 --steps 2

--kernel picks branch (the branch-parallel kernel, a barrier per substep), branch-warp (one-warp
blocks), thread (the specialised thread-per-environment kernel) or generic (the library's own).
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from paper_2502_08844_b300 import core, flops, workloads as W

CONFIG = {"cartpole": 0, "quadruped": 1, "hand": 2, "hand_elliptic": 2, "humanoid": 3}


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="quadruped", choices=sorted(CONFIG))
    ap.add_argument("--envs", type=int, default=256)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--kernel", default="branch", choices=["branch", "branch-warp", "thread", "generic"])
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    m = W.model(a.workload)
    cfg, n = CONFIG[a.workload], a.envs
    batch = core.Batch([(core.CompiledModel(m), n)])
    if a.kernel != "generic":
        batch.specialize(branch=a.kernel.startswith("branch"), warp_blocks=a.kernel == "branch-warp")
    st = core.State(batch, dev)
    ld = st.ld
    q0, v0 = W.initial_state(m, cfg, n)
    st.qpos.copy_(torch.from_numpy(core.to_soa(q0, ld, batch.nq_max)))
    st.qvel.copy_(torch.from_numpy(core.to_soa(v0, ld, batch.nv_max)))
    T = a.warmup + a.steps
    U = np.zeros((T, max(batch.nu_max, 1), ld), np.float32)
    U[:, :m.nu, :n] = W.actions(m, cfg, n, 0, T).transpose(0, 2, 1)
    ctrl = torch.from_numpy(U).to(dev)
    for t in range(a.warmup):
        core.step(batch, st, ctrl[t], m.n_substeps)
    stats = st.enable_stats()
    fm = flops.flop_model(m)
    k = batch.kernel()
    for t in range(a.steps):
        stats.zero_()
        core.step(batch, st, ctrl[a.warmup + t], m.n_substeps)
        torch.cuda.synchronize()
        iters, rows, rows_iters = (int(x) for x in stats[:, :n].to(torch.int64).sum(dim=1).cpu().numpy())
        print(json.dumps({"launch": a.warmup + t, "workload": "%s-%d" % (a.workload, n), "kernel": k["kernel"],
                          "barrier_per_substep": k["barrier_per_substep"], "substeps": n * m.n_substeps,
                          "sum_rows": rows, "sum_iters": iters, "sum_rows_iters": rows_iters,
                          "counted_flops": fm.substeps(n * m.n_substeps, rows, iters, rows_iters)}))


if __name__ == "__main__":
    main()
