"""B300-native batched rigid-body physics step (the hot path under MuJoCo Playground's
training loop, arXiv 2502.08844).

    from paper_2502_08844_b300 import workloads, core
    m = core.CompiledModel(workloads.quadruped())
    batch = core.Batch([(m, 8192)])
    state = core.State(batch)
    core.step(batch, state, ctrl, n_substeps=5)

`workloads` describes the synthetic models and seeded inputs; `core` wraps the C ABI of the
CUDA library (include/pg.h).  Importing `core` requires the built `libpg.so`.
"""
