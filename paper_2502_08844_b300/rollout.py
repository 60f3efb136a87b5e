"""Rollouts captured in CUDA graphs, and the launch autotuner.

A rollout of T control steps is T launches of the fused step kernel (one per control step,
each running its model's substeps on chip).  Capturing them in a CUDA graph removes the
per-launch host cost, which matters for small batches and short steps.

The autotuner picks, per batch composition, the kernel and the launch shape:

* the kernel: the branch-parallel one (a thread per environment and branch) in blocks that meet
  at a barrier every substep or in one-warp blocks, where some model of the batch qualifies;
  the model-specialised thread-per-environment kernel; or the library's generic kernel;
* the environments per block of the thread-per-environment kernels (one environment per
  thread; a block holds up to 8 warps of `soa` environments each, `soa` fixed per model by its
  shared-memory workspace): one wave over all SMs, or multiples of 16 around one and two waves
  whose workspace fits shared memory.

It times every candidate on the device, on the kernels that will run, and caches the fastest
per (model tables, counts, GPU name) in a JSON file.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Dict, List, Optional, Sequence, Tuple

import torch

from . import core

_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_2502_08844_b300", "autotune.json")


class GraphRollout:
    """T control steps of `pg_step` on fixed buffers, captured once and replayed."""

    def __init__(self, batch: core.Batch, state: core.State, ctrl: torch.Tensor, n_substeps: int = 0):
        assert ctrl.dim() == 3 and ctrl.shape[2] == state.ld, "ctrl is [T, nu_max, ld]"
        self.batch, self.state, self.ctrl, self.n_substeps = batch, state, ctrl, n_substeps
        self.T = ctrl.shape[0]
        self.graph: Optional[torch.cuda.CUDAGraph] = None

    def run_eager(self) -> None:
        for t in range(self.T):
            core.step(self.batch, self.state, self.ctrl[t], self.n_substeps)

    def capture(self) -> None:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):   # one eager pass on the side stream before capture
            pass
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run_eager()

    def replay(self) -> None:
        if self.graph is None:
            self.capture()
        self.graph.replay()


def _key(models: Sequence[core.CompiledModel], counts: Sequence[int]) -> str:
    h = hashlib.sha256()
    for m, n in zip(models, counts):
        s = m.sizes
        h.update(repr((m.src.name, s.nq, s.nv, s.nbody, s.nslot, s.nrow_max, s.workspace_bytes, int(n))).encode())
    return h.hexdigest()[:24] + "@" + torch.cuda.get_device_name()


def _load() -> dict:
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _save(d: dict) -> None:
    try:
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        with open(_CACHE, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
    except OSError:
        pass


KERNELS = ("branch", "branch-warp", "thread", "generic")
SMEM_PER_BLOCK = 227 * 1024


def _up16(x: int) -> int:
    return max(16, (x + 15) // 16 * 16)


def candidate_shapes(models: Sequence[core.CompiledModel], counts: Sequence[int], sms: int) -> List[int]:
    """envs-per-block candidates of the thread-per-environment kernels: 0 (one wave over all SMs,
    the library default), 16, 32, 64, 128 and the multiples of 16 nearest one and two waves, each
    no more than 256 (8 warps) and with the largest model's workspace fitting shared memory."""
    ws = max(max(m.sizes.workspace_bytes for m in models), 1)
    fit = min(256, SMEM_PER_BLOCK // ws // 16 * 16)
    total = max(sum(counts), 1)
    wave = -(-total // sms)
    cands = {16, 32, 64, 128, _up16(wave), _up16(-(-wave // 2))}
    return [0] + sorted(e for e in cands if 16 <= e <= fit)


def candidates(models: Sequence[core.CompiledModel], counts: Sequence[int], sms: int,
               kernels: Sequence[str] = KERNELS) -> List[Tuple[str, int]]:
    """(kernel, envs per block) pairs to time; the branch-parallel kernels only where some model
    qualifies.  The shape sets the thread kernels' environments per block and the barrier-launch
    branch kernel's (its warps a block: envs / environments per warp)."""
    shapes = candidate_shapes(models, counts, sms)
    branch = any(m.branch_plan()["branch"] for m in models)
    out = []
    for k in kernels:
        if k.startswith("branch") and not branch:
            continue
        # one-warp blocks take no shape of their own (the shape then applies to thread parts only)
        out += [(k, e) for e in (shapes if k != "branch-warp" or len(models) > 1 else [0])]
    return out


def make_batch(parts: Sequence[Tuple[core.CompiledModel, int]], choice: Tuple[str, int]) -> core.Batch:
    """The batch of `parts` compiled for an autotuner choice (kernel, envs per block)."""
    kernel, e = choice
    batch = core.Batch(parts, envs_per_cta=e)
    if kernel != "generic":
        batch.specialize(branch=kernel.startswith("branch"), warp_blocks=kernel == "branch-warp")
    return batch


def autotune(parts: Sequence[Tuple[core.CompiledModel, int]], n_substeps: int = 0, steps: int = 4,
             use_cache: bool = True, kernels: Sequence[str] = KERNELS) -> Tuple[str, int]:
    """The fastest (kernel, envs per block) for this batch composition (make_batch builds it).
    Run-time compilations happen here, once per model and kernel (cached on disk)."""
    models = [m for m, _ in parts]
    counts = [n for _, n in parts]
    key = _key(models, counts) + "/" + ",".join(kernels)
    cache = _load() if use_cache else {}
    if isinstance(cache.get(key), list):
        return (str(cache[key][0]), int(cache[key][1]))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    best, best_t = ("generic", 0), float("inf")
    for choice in candidates(models, counts, sms, kernels):
        try:
            batch = make_batch(parts, choice)
        except Exception:
            continue
        st = core.State(batch)
        # a plausible configuration: every model's reference pose (or zeros)
        for m, o, n in zip(models, batch.env_off, counts):
            if m.src.qpos_init is not None:
                st.qpos[:m.nq, o:o + n] = torch.from_numpy(m.src.qpos_init).to(st.qpos)[:, None]
        ctrl = torch.zeros((max(batch.nu_max, 1), st.ld), device="cuda")
        for _ in range(2):
            core.step(batch, st, ctrl, n_substeps)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            core.step(batch, st, ctrl, n_substeps)
        b.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(b)
        if t < best_t:
            best, best_t = choice, t
    cache[key] = list(best)
    if use_cache:
        _save(cache)
    return best
