"""Benchmark of the batched physics step on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload quadruped|cartpole]

One bench step = one control step (n_substeps physics substeps: FK, CRBA, LDL^T, RNEA,
collision, Jacobians, Newton solve, PD actuation, semi-implicit Euler) of every environment.
Default workload: 8192 synthetic quadrupeds, 5 substeps of 4 ms, Newton cap 4, control
targets standing pose + U(+-0.3) rad per step, K = 1000 control steps.  Prints one JSON line.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on the launching
stream; L2 is flushed (a 256 MB write) between timed steps outside the events; barrier +
synchronize around the timed region; max over ranks.  Under torchrun every rank runs its own
independent replica (envs are independent: weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2502_08844_b300 import workloads as W  # noqa: E402
from paper_2502_08844_b300 import flops as FL  # noqa: E402

METRIC = "env-steps/s on 1 B300 (quadruped, 8192 envs), % roofline; adjoint/forward time"
CONFIG_OF = {"quadruped": (1, 8192), "cartpole": (0, 256)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "pg_bench_clocks_%d_rank%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def replica_env0(rank: int, n_per_rank: int) -> int:
    """First global environment index of a rank: ranks step contiguous, disjoint env ranges of
    one job (their seeded inputs are those envs' own), no data-path exchange."""
    return rank * n_per_rank


def whole_job_rate(local_seconds: float, ws: int, n_per_rank: int, steps: int, dist=None):
    """(env-steps/s of the whole job, seconds) over all ranks: every rank's env-steps over the
    slowest rank's timed region (MAX all-reduce of the seconds when ws > 1)."""
    secs = float(local_seconds)
    if ws > 1:
        import torch
        t = torch.tensor([secs], dtype=torch.float64)
        if torch.cuda.is_available() and dist.get_backend() == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        secs = float(t.item())
    return ws * n_per_rank * steps / secs, secs


def kernel_source_hash() -> str:
    """sha256 (first 16 hex digits) of the step kernels' sources (the generic, the run-time
    specialised and the branch-parallel builds): device functions, kernel bodies, kernels,
    translation unit, specialiser, branch plan and internal layout header, in that order."""
    h = hashlib.sha256()
    for f in ("step_device.cuh", "step_kernel_body.cuh", "step_kernels.cuh", "step.cu", "specialize.cpp",
              "branch_body.cuh", "branch.cpp", "pg_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2502_08844_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def kernel_traffic(workload: str):
    """DRAM bytes per launch from a committed ncu summary, valid only for the current kernel source."""
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    ent = d.get(workload)
    if not ent or ent.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


def cpu_sample_envs() -> int:
    """Environments of the oracle's timed sample (the CPU baseline and the reference arm): 16 per
    host core, at least 256."""
    return max(256, 16 * (os.cpu_count() or 1))


def cpu_baseline(model: W.Model, cfg: int, n_envs: int, budget_s: float = 10.0, chunk: int = 10):
    """The FP64 oracle (its -O3 -march=native build) on all host cores, on a bounded sample of the
    workload: cpu_sample_envs() environments, chunks of `chunk` control steps per call, until
    budget_s seconds have passed."""
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    om = O.OracleModel(model, native=True)
    n = min(n_envs, cpu_sample_envs())
    q, v = W.initial_state(model, cfg, n)
    warm = None
    steps, t0 = 0, time.time()
    q = q.astype(np.float64); v = v.astype(np.float64)
    while True:
        U = W.actions(model, cfg, n, steps, chunk)
        q, v, warm, _ = om.rollout(q, v, U, model.n_substeps, qacc_warm=warm, nthreads=cores)
        steps += chunk
        if time.time() - t0 >= budget_s:
            break
    dt = time.time() - t0
    return {"value": n * steps / dt, "unit": "env-steps/s", "cores": cores, "kind": "oracle",
            "sample": "%d envs x %d control steps (%d substeps each, %d-step calls) of the %s workload, FP64 "
                      "(-O3 -march=native), %d threads" % (n, steps, model.n_substeps, chunk, model.name, cores)}


def measure_mixed(dev, steps: int = 200, specialize: bool = True):
    """Mixed-model batch: 4096 cartpoles + 4096 quadrupeds + 2048 humanoids (each env with its
    own model's timestep and substeps), a 200-step rollout captured in a CUDA graph.  Specialised:
    the kernel and launch shape the autotuner picks among the branch-parallel, specialised
    thread-per-environment and generic kernels; generic: the one launch of the library's kernel
    over every model, at the autotuner's shape for that kernel."""
    import torch
    from paper_2502_08844_b300 import core, rollout
    comp = [("cartpole", 0, 4096), ("quadruped", 1, 4096), ("humanoid", 3, 2048)]
    models = [(core.CompiledModel(W.model(nm)), n) for nm, _, n in comp]
    choice = rollout.autotune(models, kernels=rollout.KERNELS if specialize else ("generic",))
    batch = rollout.make_batch(models, choice)
    epc = choice[1]
    specialize = choice[0] != "generic"
    st = core.State(batch, dev)
    ld = st.ld
    Q = np.zeros((batch.nq_max, ld), np.float32)
    V = np.zeros((batch.nv_max, ld), np.float32)
    U = np.zeros((steps, max(batch.nu_max, 1), ld), np.float32)
    o = 0
    for (nm, cfg, n), (cm, _) in zip(comp, models):
        m = cm.src
        q0, v0 = W.initial_state(m, cfg, n)
        Q[:m.nq, o:o + n] = q0.T
        V[:m.nv, o:o + n] = v0.T
        U[:, :m.nu, o:o + n] = W.actions(m, cfg, n, 0, steps).transpose(0, 2, 1)
        o += n
    st.qpos.copy_(torch.from_numpy(Q)); st.qvel.copy_(torch.from_numpy(V))
    ctrl = torch.from_numpy(U).to(dev)
    g = rollout.GraphRollout(batch, st, ctrl, 0)
    g.capture()
    st.qpos.copy_(torch.from_numpy(Q)); st.qvel.copy_(torch.from_numpy(V)); st.qacc_warm.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(); g.replay(); b.record()
    torch.cuda.synchronize()
    t_graph = a.elapsed_time(b) / 1e3
    st.qpos.copy_(torch.from_numpy(Q)); st.qvel.copy_(torch.from_numpy(V)); st.qacc_warm.zero_()
    torch.cuda.synchronize()
    a.record(); g.run_eager(); b.record()
    torch.cuda.synchronize()
    t_eager = a.elapsed_time(b) / 1e3
    n_tot = sum(n for _, _, n in comp)
    k = batch.kernel()
    return {"value": n_tot * steps / t_graph, "unit": "env-steps/s", "eager_value": n_tot * steps / t_eager,
            "kernel": ("model-specialised: one kernel per model over its own environments, back to back; the "
                       "branch-parallel kernel for %d of the %d models" % (k["branch_parts"], len(comp))) if specialize
                      else "generic (one body shared by the batch's models)",
            "composition": {nm: n for nm, _, n in comp}, "steps": steps, "cuda_graph": True,
            "autotuned": {"kernel": choice[0], "envs_per_cta": epc or "default (one wave)"},
            "launches": steps * (len(comp) if specialize else 1)}


def measure_env_layer(dev, n: int = 8192, steps: int = 200, specialize: bool = True):
    """The locomotion task around the step (pg_env_step: joint targets, physics, reward table,
    termination, auto-reset and observation) against the plain step on the same 8192 quadrupeds,
    same policy actions and commands.  Specialised: the substeps on the branch-parallel kernel
    between a targets launch and an end-of-step launch, against the plain branch-parallel step.
    Time per control step with CUDA events around `steps` back-to-back launches (inputs are
    device-resident; the state and task arrays, a few MB, stay in L2)."""
    import torch
    from paper_2502_08844_b300 import core
    m = W.quadruped()
    cm = core.CompiledModel(m)
    batch = core.Batch([(cm, n)])
    if specialize:
        batch.specialize()
    task = core.Task(cm, W.quadruped_task(episode_length=1000))
    st = core.State(batch, dev)
    ld = st.ld
    q0, v0 = W.initial_state(m, 1, n)
    Q0 = torch.from_numpy(core.to_soa(q0, ld, batch.nq_max)).to(dev)
    V0 = torch.from_numpy(core.to_soa(v0, ld, batch.nv_max)).to(dev)
    cmd = torch.from_numpy(core.to_soa(W.commands(1, n), ld, 3)).to(dev)
    A = np.zeros((steps, m.nu, ld), np.float32)
    A[:, :, :n] = W.policy_actions(m, 1, n, 0, steps).transpose(0, 2, 1)
    act = torch.from_numpy(A).to(dev)
    ctrl = torch.from_numpy(task.src.q_default[None, :, None] + task.src.action_scale * A).to(dev).contiguous()
    ts = torch.zeros((task.state_rows, ld), device=dev)
    obs = torch.zeros((task.nobs, ld), device=dev)
    rew, done, trunc = (torch.zeros(ld, device=dev) for _ in range(3))

    def env_run():
        core.env_reset(batch, task, st, ts, Q0, V0, cmd, obs)
        for t in range(steps):
            core.env_step(batch, task, st, ts, act[t], cmd, Q0, V0, 0, obs, rew, done, trunc)

    def plain_run():
        core.reset(batch, st, Q0, V0)
        for t in range(steps):
            core.step(batch, st, ctrl[t], 0)

    def timed(f):
        f()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(); f(); b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    t_env, t_plain = timed(env_run), timed(plain_run)
    return {"value": n * steps / t_env, "unit": "env-steps/s", "plain_step_value": n * steps / t_plain,
            "overhead": t_env / t_plain - 1.0, "envs": n, "steps": steps, "episode_length": 1000,
            "kernel": batch.kernel()["kernel"] if specialize else "generic",
            "launches_per_env_step": 3 if specialize and batch.kernel()["kernel"] == "branch-parallel" else 1,
            "note": "pg_env_step vs pg_step on identical targets (absolute mapping); reset launch included"}


def measure_rough_terrain(dev, n: int = 8192, steps: int = 200, specialize: bool = True):
    """The quadruped on rough terrain (an 81 x 81 heightfield of gradient noise instead of the
    floor plane), 8192 environments, the bench workload's actions: env-steps/s of the step with
    heightfield contacts, CUDA events around `steps` launches (the 26 KB elevation grid stays in
    L1/L2; the state is device-resident)."""
    import torch
    from paper_2502_08844_b300 import core
    m = W.quadruped_rough()
    batch = core.Batch([(core.CompiledModel(m), n)])
    if specialize:
        batch.specialize()
    st = core.State(batch, dev)
    ld = st.ld
    q0, v0 = W.initial_state(m, 1, n)
    Q0 = torch.from_numpy(core.to_soa(q0, ld, batch.nq_max)).to(dev)
    V0 = torch.from_numpy(core.to_soa(v0, ld, batch.nv_max)).to(dev)
    U = np.zeros((steps, m.nu, ld), np.float32)
    U[:, :, :n] = W.actions(m, 1, n, 0, steps).transpose(0, 2, 1)
    ctrl = torch.from_numpy(U).to(dev)

    def run():
        core.reset(batch, st, Q0, V0)
        for t in range(steps):
            core.step(batch, st, ctrl[t], 0)

    run()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(); run(); b.record()
    torch.cuda.synchronize()
    t = a.elapsed_time(b) / 1e3
    return {"value": n * steps / t, "unit": "env-steps/s", "envs": n, "steps": steps,
            "terrain": "81 x 81 heightfield, 0.1 m cells, 6 cm relief", "kernel": batch.kernel()["kernel"]}


def measure_dr(dev, n: int = 8192, steps: int = 200, specialize: bool = True):
    """pg_step_dr on the bench workload (8192 quadrupeds) with every environment's parameters drawn
    as in workloads.randomized_params (friction, payload, centres of mass, armature, calibration,
    gains and link masses), against pg_step on the same batch: CUDA events around `steps` launches
    each, the state device-resident."""
    import torch
    from paper_2502_08844_b300 import core
    m = W.quadruped()
    batch = core.Batch([(core.CompiledModel(m), n)])
    if specialize:
        batch.specialize()
    st = core.State(batch, dev)
    ld = st.ld
    q0, v0 = W.initial_state(m, 1, n)
    Q0 = torch.from_numpy(core.to_soa(q0, ld, batch.nq_max)).to(dev)
    V0 = torch.from_numpy(core.to_soa(v0, ld, batch.nv_max)).to(dev)
    U = np.zeros((steps, m.nu, ld), np.float32)
    U[:, :, :n] = W.actions(m, 1, n, 0, steps).transpose(0, 2, 1)
    ctrl = torch.from_numpy(U).to(dev)
    P = W.randomized_params(m, 1, n)
    params = torch.from_numpy(core.to_soa(P, ld, P.shape[1])).to(dev)

    def run(dr):
        core.reset(batch, st, Q0, V0)
        for t in range(steps):
            if dr:
                core.step_dr(batch, st, ctrl[t], params, 0)
            else:
                core.step(batch, st, ctrl[t], 0)

    def timed(dr):
        run(dr)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(); run(dr); b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    t_dr, t_plain = timed(True), timed(False)
    k = batch.kernel()
    return {"value": n * steps / t_dr, "unit": "env-steps/s", "envs": n, "steps": steps,
            "plain_step_value": n * steps / t_plain, "overhead": t_dr / t_plain - 1.0,
            "nrand": int(P.shape[1]),
            "kernel": ("branch-parallel (pg_step_branch_dr)" if k["branch_dr"]
                       else "thread-per-environment (%s)" % k["kernel"])}


def measure_pixels(dev, n: int = 8192, steps: int = 50):
    """Pixel observations of the cartpole: 8192 environments, one 64 x 64 RGB (uint8) ray-traced
    image each per control step (pg_render after pg_step), the paper's CartpoleBalance-from-pixels
    setting (Sec. 5; App. "Madrona benchmark").  Reports physics + render env-steps/s, physics
    alone, and the frames/s the renders add (the difference of the two), CUDA events around
    `steps` steps from the same initial state."""
    import torch
    from paper_2502_08844_b300 import core
    m = W.cartpole_pixels()
    scene = W.cartpole_scene()
    batch = core.Batch([(core.CompiledModel(m), n)])
    batch.specialize()
    st = core.State(batch, dev)
    ld = st.ld
    q0, v0 = W.initial_state(m, 0, n)
    Q0 = torch.from_numpy(core.to_soa(q0, ld, batch.nq_max)).to(dev)
    V0 = torch.from_numpy(core.to_soa(v0, ld, batch.nv_max)).to(dev)
    U = np.zeros((steps, 1, ld), np.float32)
    U[:, :, :n] = W.actions(m, 0, n, 0, steps).transpose(0, 2, 1)
    ctrl = torch.from_numpy(U).to(dev)
    px = torch.zeros((n, scene.height, scene.width, 3), dtype=torch.uint8, device=dev)

    def timed(f):
        f()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(); f(); b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    def step_only():
        core.reset(batch, st, Q0, V0)
        for t in range(steps):
            core.step(batch, st, ctrl[t], 1)

    def step_and_render():
        core.reset(batch, st, Q0, V0)
        for t in range(steps):
            core.step(batch, st, ctrl[t], 1)
            core.render(batch, st, scene, px)

    # every loop starts from the same state and sees the same sequence of states
    t_s, t_sr = timed(step_only), timed(step_and_render)
    t_r = max(t_sr - t_s, 1e-9)
    rays = n * scene.width * scene.height
    return {"frames_per_s": n * steps / t_r, "env_steps_per_s_with_pixels": n * steps / t_sr,
            "env_steps_per_s_physics_only": n * steps / t_s,
            "ms_per_render": 1e3 * t_r / steps, "primary_rays_per_s": rays * steps / t_r,
            "resolution": [scene.width, scene.height], "envs": n, "steps": steps,
            "output_bytes_per_frame": 3 * rays,
            "paper_context": "cartpole with pixels ~403,000 steps/s (Madrona + MJX, Sec. 5; other hardware)"}


def run_reference(args):
    """Reference arm: the FP64 oracle as it stands (its -O3 -march=native build), timed on the
    host cores on the CPU baseline's sample shape: cpu_sample_envs() environments of the workload,
    the W warm-up control steps in one call, then the K timed control steps in one call."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cfg, n_total = CONFIG_OF[args.workload]
    m = W.model(args.workload)
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    om = O.OracleModel(m, native=True)
    n = min(n_total, cpu_sample_envs())
    q, v = W.initial_state(m, cfg, n)
    q = q.astype(np.float64); v = v.astype(np.float64)
    q, v, warm, _ = om.rollout(q, v, W.actions(m, cfg, n, 0, args.warmup), m.n_substeps, nthreads=cores)
    U = W.actions(m, cfg, n, args.warmup, args.steps)
    t0 = time.time()
    q, v, warm, _ = om.rollout(q, v, U, m.n_substeps, qacc_warm=warm, nthreads=cores)
    dt = time.time() - t0
    val = n * args.steps / dt
    line = {"metric": METRIC, "value": val, "unit": "env-steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "%s-%d" % (args.workload, n_total), "sample_envs_per_step": n,
                       "substeps": m.n_substeps, "newton_cap": m.iterations},
            "impl": "reference",
            "cpu_baseline": {"value": val, "unit": "env-steps/s", "cores": cores, "kind": "oracle",
                             "sample": "%d envs x %d control steps in one call, FP64 oracle (-O3 -march=native), "
                                       "%d threads" % (n, args.steps, cores)},
            "e2e": {"value": val, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def measure_adjoint(dev, n: int = 4096, steps: int = 64, segment: int = 8, reps: int = 3, specialize: bool = True,
                    branch: bool = True):
    """Full rollout gradient against the forward rollout on the adjoint workload: 4096
    quadrupeds, 64 control steps, loss sum_t (z_t - 0.27)^2 + |v_t - (0.5, 0, 0)|^2 of the torso
    height and linear velocity, gradients with respect to the initial state, all 64 x 12
    controls and the per-environment masses, damping and kp, checkpoints every 8 steps.  The
    gradient's time covers the checkpointed forward pass, the loss and the backward sweep."""
    import torch
    from paper_2502_08844_b300 import adjoint, core
    m = W.quadruped()
    cm = core.CompiledModel(m)
    batch = core.Batch([(cm, n)])
    if specialize:   # forward, tape replay and reverse sweep compiled for the model
        batch.specialize(branch=branch)
    st = core.State(batch, dev)
    ld = st.ld
    q0, v0 = W.initial_state(m, 4, n)
    U = W.actions(m, 4, n, 0, steps)
    Q0 = torch.from_numpy(core.to_soa(q0, ld, batch.nq_max)).to(dev)
    V0 = torch.from_numpy(core.to_soa(v0, ld, batch.nv_max)).to(dev)
    Us = np.zeros((steps, batch.nu_max, ld), np.float32)
    Us[:, :m.nu, :n] = U.transpose(0, 2, 1)
    ctrl = torch.from_numpy(Us).to(dev)
    params = adjoint.param_values(batch, ld, dev)
    zs = torch.zeros((batch.nq_max, 1), device=dev); zs[2] = 0.27
    vs = torch.zeros((batch.nv_max, 1), device=dev); vs[0] = 0.5
    wq = torch.zeros((batch.nq_max, 1), device=dev); wq[2] = 1.0
    wv = torch.zeros((batch.nv_max, 1), device=dev); wv[:3] = 1.0

    def forward():
        st.qpos.copy_(Q0); st.qvel.copy_(V0); st.qacc_warm.zero_()
        for t in range(steps):
            core.step(batch, st, ctrl[t], 0)

    def gradient():
        q = Q0.clone().requires_grad_(); v = V0.clone().requires_grad_()
        u = ctrl.clone().requires_grad_(); p = params.clone().requires_grad_()
        Q, V = adjoint.rollout(batch, q, v, u, p, 0, segment)
        loss = (wq * (Q[:, :, :n] - zs) ** 2).sum() + (wv * (V[:, :, :n] - vs) ** 2).sum()
        loss.backward()
        return loss

    def timed(f):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        f()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    gradient(); forward()   # warm-up (the adjoint's scratch is allocated on its first call)
    tf = min(timed(forward) for _ in range(reps))
    tg = min(timed(gradient) for _ in range(reps))
    k = batch.kernel()
    return {"ratio": tg / tf, "forward_ms": tf, "gradient_ms": tg, "envs": n, "steps": steps, "segment": segment,
            "newton_cap": m.iterations,
            "kernels": ("forward and tape replay: %s; reverse sweep: model-specialised thread-per-environment"
                        % k["kernel"]) if specialize else "generic",
            "note": "gradient = checkpointed forward + loss + backward sweep"}


# the other workload configurations, each timed on its own (model, input config, envs, control
# steps timed): the cartpole (256 envs; 1000 steps as configured), the hand with the pyramidal
# and the elliptic cone (8192 envs; 50 of the configured 500 control steps of 10 substeps), the
# humanoid at the mixed batch's count (2048 envs)
WORKLOADS = [("cartpole-256", "cartpole", 0, 256, 1000), ("hand-8192", "hand", 2, 8192, 50),
             ("hand_elliptic-8192", "hand_elliptic", 2, 8192, 50), ("humanoid-2048", "humanoid", 3, 2048, 200)]


def roofline_alu(m: W.Model, n: int, steps: int, sums, mean_launch_s: float, dev):
    """ALU roofline of launches of the step: counted flops (flops.py) over the CUDA-core FP32 peak."""
    import torch
    fm = FL.flop_model(m)
    flops_launch = fm.substeps(n * m.n_substeps * steps, sums[1], sums[0], sums[2]) / steps
    peaks, src = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    peak = FL.fp32_peak_tflops(props.multi_processor_count, sm_mhz)
    achieved = flops_launch / mean_launch_s / 1e12
    bytes_launch = n * 4 * (2 * (m.nq + 2 * m.nv) + m.nu)
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": "%d SMs x 128 FP32 lanes x 2 x sm_max_mhz %.0f (%s)" % (props.multi_processor_count, sm_mhz,
                                                                                   src),
            "flops_per_launch": flops_launch, "flops_source": "counted FP64 oracle, per-substep fit (flop_counts.json)",
            "algorithmic_bytes_per_launch": bytes_launch,
            "hbm_frac": bytes_launch / mean_launch_s / 1e9 / float(peaks.get("hbm_gbs", 6400.0)),
            "newton_iters_per_substep": float(sums[0]) / (n * m.n_substeps * steps),
            "rows_per_substep": float(sums[1]) / (n * m.n_substeps * steps)}


def measure_workload(dev, name: str, cfg: int, n: int, steps: int, branch: bool = True, warmup: int = 3,
                     warp_blocks: bool = False):
    """Env-steps/s of one workload (its own launches, CUDA events around `steps` back-to-back
    control steps; inputs device-resident) and its ALU roofline."""
    import torch
    from paper_2502_08844_b300 import core
    m = W.model(name)
    batch = core.Batch([(core.CompiledModel(m), n)])
    batch.specialize(branch=branch, warp_blocks=warp_blocks)
    st = core.State(batch, dev)
    ld = st.ld
    q0, v0 = W.initial_state(m, cfg, n)
    st.qpos.copy_(torch.from_numpy(core.to_soa(q0, ld, batch.nq_max)))
    st.qvel.copy_(torch.from_numpy(core.to_soa(v0, ld, batch.nv_max)))
    U = np.zeros((warmup + steps, max(batch.nu_max, 1), ld), np.float32)
    U[:, :m.nu, :n] = W.actions(m, cfg, n, 0, warmup + steps).transpose(0, 2, 1)
    ctrl = torch.from_numpy(U).to(dev)
    for t in range(warmup):
        core.step(batch, st, ctrl[t], m.n_substeps)
    stats = st.enable_stats()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for t in range(steps):
        core.step(batch, st, ctrl[warmup + t], m.n_substeps)
    b.record()
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    sums = stats[:, :n].to(torch.int64).sum(dim=1).cpu().numpy()
    k = batch.kernel()
    return {"value": n * steps / sec, "unit": "env-steps/s", "envs": n, "steps": steps, "substeps": m.n_substeps,
            "newton_cap": m.iterations, "ms_per_step": 1e3 * sec / steps,
            "kernel": k["kernel"] + ("" if k["kernel"] != "branch-parallel" else
                                     " (%d lanes per environment, %d branches, %s)" % (
                                         k["lanes_per_env"], k["branches"],
                                         "barrier per substep" if k["barrier_per_substep"] else "one-warp blocks")),
            "branch_kernel_not_used_because": k["reason"] or None,
            "roofline": roofline_alu(m, n, steps, sums, sec / steps, dev)}


def kernel_requests(args, single: bool) -> list:
    """(model, environments, envs_per_cta, branch) of every model this run specialises: the
    headline workload and, on one GPU, the sub-measurements' models (kernel_cache requests)."""
    cfg, n = CONFIG_OF[args.workload]
    reqs = [] if args.generic_kernel else [(W.model(args.workload), n, args.envs_per_cta, not args.thread_kernel)]
    if single and not args.no_workloads:
        reqs += [(W.model(nm), n_w, 0, True) for _, nm, _, n_w, _ in WORKLOADS]
    if single and not args.no_mixed:   # the autotuner's candidates: one-wave shapes and fixed ones
        reqs += [(W.model(nm), n_m, e, True) for nm, n_m in (("cartpole", 4096), ("quadruped", 4096),
                                                            ("humanoid", 2048)) for e in (0, 16)]
    if single and not args.no_env:
        reqs += [(W.quadruped(), 8192, 0, True), (W.quadruped_rough(), 8192, 0, True),
                 (W.cartpole_pixels(), 8192, 0, True)]
    if single and not args.no_adjoint:
        reqs += [(W.quadruped(), 4096, 0, True)]
    return reqs


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2502_08844_b300 import core

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # the specialised kernels of every model this run uses, compiled up front in parallel host
    # threads (NVRTC; cached on disk); each specialisation below then loads its cubin
    try:
        from paper_2502_08844_b300 import kernel_cache
        pre = kernel_cache.precompile(kernel_requests(args, ws == 1), cache_dir=None)
    except Exception as e:   # each specialisation then compiles its own kernels, as without it
        pre = {"models": 0, "wall_s": 0.0, "failed": [str(e)]}
    cfg, n = CONFIG_OF[args.workload]
    m = W.model(args.workload)
    cm = core.CompiledModel(m)
    batch = core.Batch([(cm, n)], envs_per_cta=args.envs_per_cta)
    kernel = "generic"
    if not args.generic_kernel:
        try:
            # NVRTC, cached; seconds on a first compile (outside the timed region); the
            # branch-parallel kernel where the model qualifies, else the thread-per-environment one
            batch.specialize(branch=not args.thread_kernel)
            k = batch.kernel()
            kernel = ("branch-parallel (run-time compiled; %d lanes per environment, %d branches; %s)"
                      % (k["lanes_per_env"], k["branches"],
                         "one wave of blocks whose warps start each substep together" if k["barrier_per_substep"]
                         else "blocks of one warp") if k["kernel"] == "branch-parallel"
                      else "model-specialised (run-time compiled)")
        except Exception as e:   # keeps the generic kernel; reported in the line
            kernel = "generic (specialisation failed: %s)" % str(e).splitlines()[0][:200]
    state = core.State(batch, dev)
    env0 = replica_env0(rank, n)
    q0, v0 = W.initial_state(m, cfg, n, env0)
    ld = state.ld
    state.qpos.copy_(torch.from_numpy(core.to_soa(q0, ld, batch.nq_max)))
    state.qvel.copy_(torch.from_numpy(core.to_soa(v0, ld, batch.nv_max)))
    T = args.warmup + args.steps
    U = W.actions(m, cfg, n, 0, T, env0)                                # [T, n, nu]
    Usoa = np.zeros((T, max(batch.nu_max, 1), ld), np.float32)
    Usoa[:, :m.nu, :n] = U.transpose(0, 2, 1)
    ctrl = torch.from_numpy(Usoa).to(dev)
    stream = torch.cuda.current_stream()
    for t in range(args.warmup):
        core.step(batch, state, ctrl[t], m.n_substeps)
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stats = state.enable_stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    # the clock samples (every 20 ms) need the GPU under this load for longer than a short timed
    # region lasts: untimed steps of the same workload from a copy of the state fill about 0.5 s
    # just before it (the timed steps start from the warmed-up state itself)
    side = core.State(batch, dev)
    side.qpos.copy_(state.qpos); side.qvel.copy_(state.qvel); side.qacc_warm.copy_(state.qacc_warm)
    a0, b0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    core.step(batch, side, ctrl[0], m.n_substeps)
    b0.record(stream)
    torch.cuda.synchronize()
    n_fill = int(min(20000, 0.5e3 / max(a0.elapsed_time(b0), 1e-3)))
    for k in range(n_fill):
        core.step(batch, side, ctrl[k % T], m.n_substeps)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.time()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        core.step(batch, state, ctrl[args.warmup + k], m.n_substeps)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    wall = time.time() - wall0
    ck = clocks.stop()
    if ck is not None:
        ck["window"] = "%d untimed steps of the workload just before the timed region, and the timed region" % n_fill
    times = [a.elapsed_time(b) for a, b in ev]          # ms per launch
    dev_s = sum(times) / 1e3
    st = stats[:, :n].to(torch.int64).sum(dim=1).cpu().numpy()
    status = state.status.cpu().numpy().view(np.uint32)
    value, dev_s = whole_job_rate(dev_s, ws, n, args.steps, dist)
    # roofline: algorithmic (counted) FP32 flops per launch / mean launch time, against the CUDA-core peak
    roof = roofline_alu(m, n, args.steps, st, statistics.mean(times) / 1e3, dev)
    roof["traffic"] = kernel_traffic(args.workload)
    # end to end through the C ABI with host buffers (pinned), every step's control upload and
    # state download inside the timed region: pg_rollout_host (transfers overlapped with the
    # steps), and pg_step_host once per step for comparison
    e2e = None
    if not args.no_e2e:
        Ke = min(args.steps, 200)
        ctrl_h = torch.from_numpy(np.ascontiguousarray(Usoa[args.warmup:args.warmup + Ke])).pin_memory()
        qh = torch.empty((Ke, batch.nq_max, ld), dtype=torch.float32).pin_memory()
        vh = torch.empty((Ke, batch.nv_max, ld), dtype=torch.float32).pin_memory()
        state.stats = None
        core.rollout_host(batch, state, ctrl_h[:2], qh[:2], vh[:2], m.n_substeps)   # staging set-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        core.rollout_host(batch, state, ctrl_h, qh, vh, m.n_substeps)
        e1.record(stream)
        torch.cuda.synchronize()
        t_e2e = e0.elapsed_time(e1) / 1e3
        e0.record(stream)
        for k in range(Ke):
            core.step_host(batch, state, ctrl_h[k], qh[k], vh[k], m.n_substeps)
        e1.record(stream)
        torch.cuda.synchronize()
        t_call = e0.elapsed_time(e1) / 1e3
        e2e = {"value": ws * n * Ke / t_e2e, "unit": "env-steps/s", "steps": Ke,
               "api": "pg_rollout_host (uploads and downloads overlapped with the steps)",
               "per_call_value": ws * n * Ke / t_call, "per_call_api": "pg_step_host once per step",
               "h2d_bytes_per_step": int(batch.nu_max * ld * 4),
               "d2h_bytes_per_step": int((batch.nq_max + batch.nv_max) * ld * 4)}
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "%s-%d" % (args.workload, n), "n_envs_per_gpu": n, "substeps": m.n_substeps,
                       "dt": m.timestep, "newton_cap": m.iterations, "cone": "pyramidal",
                       "envs_per_cta": args.envs_per_cta or "default", "kernel": kernel,
                       "l2": "flushed between timed steps (256 MB write outside the events)",
                       "wall_s_timed_region": wall,
                       "kernel_precompile": {"models": pre["models"], "wall_s": round(pre["wall_s"], 1),
                                             "failed": pre["failed"]}},
            "roofline": roof, "e2e": e2e, "gpu_launches": args.steps,
            "clocks": ck, "status_bits_seen": int(np.bitwise_or.reduce(status)) if status.size else 0,
            "adjoint_forward_ratio": None}
    # the sub-measurements characterise one GPU: the N = 1 line carries them, scaling runs skip them
    single = ws == 1
    spec = not kernel.startswith("generic")
    if single and not args.no_workloads:
        line["workloads"] = {label: measure_workload(dev, nm, cfg_w, n_w, steps_w)
                             for label, nm, cfg_w, n_w, steps_w in WORKLOADS}
        if kernel.startswith("branch"):   # the headline workload and the humanoid on the other kernels
            for nm, cfg_w, n_w in ((args.workload, cfg, n), ("humanoid", 3, 2048)):
                line["workloads"]["%s-%d branch-parallel in one-warp blocks" % (nm, n_w)] = measure_workload(
                    dev, nm, cfg_w, n_w, 200, warp_blocks=True)
                line["workloads"]["%s-%d thread-per-environment" % (nm, n_w)] = measure_workload(
                    dev, nm, cfg_w, n_w, 200, branch=False)
    if single and not args.no_mixed:
        line["mixed_batch"] = measure_mixed(dev, specialize=spec)
        if spec:
            line["mixed_batch"]["generic_kernel"] = {k: v for k, v in measure_mixed(dev, specialize=False).items()
                                                     if k in ("value", "eager_value")}
    if single and not args.no_env:
        line["env_layer"] = measure_env_layer(dev, specialize=spec)
        line["rough_terrain"] = measure_rough_terrain(dev, specialize=spec)
        line["domain_randomisation"] = measure_dr(dev, specialize=spec)
        line["pixels"] = measure_pixels(dev)
    if single and not args.no_adjoint:
        adj = measure_adjoint(dev, specialize=spec)
        line["adjoint_forward_ratio"] = adj["ratio"]
        line["adjoint"] = adj
        gen = measure_adjoint(dev, specialize=False)
        line["adjoint"]["generic_kernels"] = {"ratio": gen["ratio"], "forward_ms": gen["forward_ms"],
                                              "gradient_ms": gen["gradient_ms"]}
        thr = measure_adjoint(dev, specialize=True, branch=False)
        line["adjoint"]["thread_per_environment_kernels"] = {"ratio": thr["ratio"], "forward_ms": thr["forward_ms"],
                                                             "gradient_ms": thr["gradient_ms"]}
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(m, cfg, n)
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(CONFIG_OF), default="quadruped")
    ap.add_argument("--envs-per-cta", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-env", action="store_true", help="skip the locomotion-task measurement")
    ap.add_argument("--pixels-only", type=int, default=0, metavar="N",
                    help="only the pixel-observation measurement, on N cartpoles (for profiling the renderer)")
    ap.add_argument("--generic-kernel", action="store_true", help="skip pg_batch_specialize")
    ap.add_argument("--thread-kernel", action="store_true",
                    help="the model-specialised thread-per-environment kernel, not the branch-parallel one")
    ap.add_argument("--no-workloads", action="store_true", help="skip the other workload configurations")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.pixels_only:
        import torch
        print(json.dumps(measure_pixels(torch.device("cuda"), n=args.pixels_only, steps=max(args.steps, 1))))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
