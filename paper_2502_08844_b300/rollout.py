"""Rollouts captured in CUDA graphs, and the launch-shape autotuner.

A rollout of T control steps is T launches of the fused step kernel (one per control step,
each running its model's substeps on chip).  Capturing them in a CUDA graph removes the
per-launch host cost, which matters for small batches and short steps.

The autotuner picks the environments-per-block of a batch (the kernel runs one environment
per thread; a block holds up to 8 warps of `soa` environments each, `soa` fixed per model by its
shared-memory workspace).  It times a few candidate shapes on the device and caches the
fastest per (model tables, counts, GPU name) in a JSON file.
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


def _load() -> Dict[str, int]:
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _save(d: Dict[str, int]) -> None:
    try:
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        with open(_CACHE, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
    except OSError:
        pass


def candidate_shapes(models: Sequence[core.CompiledModel], counts: Sequence[int], sms: int) -> List[int]:
    """envs-per-block candidates: 0 (one wave over all SMs, the library default) and multiples of
    the smallest SoA width, up to what shared memory admits."""
    out = [0]
    for e in (16, 32, 48, 64, 96, 128):
        if e not in out:
            out.append(e)
    return out


def autotune(parts: Sequence[Tuple[core.CompiledModel, int]], n_substeps: int = 0, steps: int = 4,
             use_cache: bool = True) -> int:
    """Return the fastest envs_per_cta for this batch composition (0 = library default)."""
    models = [m for m, _ in parts]
    counts = [n for _, n in parts]
    key = _key(models, counts)
    cache = _load() if use_cache else {}
    if key in cache:
        return int(cache[key])
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    best, best_t = 0, float("inf")
    for e in candidate_shapes(models, counts, sms):
        try:
            batch = core.Batch(parts, envs_per_cta=e)
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
            best, best_t = e, t
    cache[key] = best
    if use_cache:
        _save(cache)
    return best
