"""CPU checks of the autotuner's host logic (rollout.candidate_shapes, rollout.candidates): which
launch shapes and kernels it times, without timing them."""
from paper_2502_08844_b300 import core, rollout
from paper_2502_08844_b300 import workloads as W


def _models(*names):
    return [core.CompiledModel(W.model(n)) for n in names]


def test_shapes_of_a_mixed_batch():
    """4096 cartpoles + 4096 quadrupeds on 148 SMs: one wave is 56 environments a block (64 as a
    multiple of 16), two waves 28 (32); the quadruped's 3.3 KB workspace caps a block at 64."""
    models = _models("cartpole", "quadruped")
    shapes = rollout.candidate_shapes(models, [4096, 4096], 148)
    assert shapes == [0, 16, 32, 64]
    ws = max(m.sizes.workspace_bytes for m in models)
    assert all(e * ws <= rollout.SMEM_PER_BLOCK and e <= 256 for e in shapes[1:])
    # with the humanoid (8.6 KB a workspace) a block holds 16 at most
    assert rollout.candidate_shapes(_models("cartpole", "quadruped", "humanoid"), [4096, 4096, 2048], 148) == [0, 16]


def test_shapes_never_exceed_what_shared_memory_holds():
    """The hand's 11 KB workspace: 16 environments a block at most."""
    hand = _models("hand")
    assert rollout.candidate_shapes(hand, [8192], 148) == [0, 16]


def test_branch_kernels_only_where_a_model_qualifies():
    cart = _models("cartpole")
    ks = {k for k, _ in rollout.candidates(cart, [4096], 148)}
    assert ks == {"thread", "generic"}
    quad = _models("quadruped")
    c = rollout.candidates(quad, [8192], 148)
    assert {k for k, _ in c} == set(rollout.KERNELS)
    # one model in one-warp blocks takes no shape of its own
    assert [e for k, e in c if k == "branch-warp"] == [0]
    mixed = _models("cartpole", "quadruped")
    c = rollout.candidates(mixed, [4096, 4096], 148)
    assert len([e for k, e in c if k == "branch-warp"]) == len(rollout.candidate_shapes(mixed, [4096, 4096], 148))
    assert all(k == "generic" for k, _ in rollout.candidates(quad, [8192], 148, ("generic",)))
