"""The seeded input generators (workloads.py) that both the CUDA path's tests and the oracle draw
from: the counter-based SplitMix64 stream against its published outputs, and the properties the
input recipe relies on (draws depend on (config, environment, index) only, so any slice of a batch
or of a rollout, and any shard of environments across ranks, sees the same inputs)."""
import numpy as np
import pytest

from paper_2502_08844_b300 import workloads as W


def test_splitmix64_matches_its_published_outputs():
    """SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
    OOPSLA 2014; the generator Vigna uses to seed xoshiro): the first outputs of the streams
    seeded with 0 and with 1234567."""
    k = np.arange(5, dtype=np.uint64)
    assert [int(x) for x in W.splitmix64(np.uint64(0), k)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC, 0x1B39896A51A8749B]
    assert [int(x) for x in W.splitmix64(np.uint64(1234567), k)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
        16408922859458223821]


def test_uniform01_takes_the_top_53_bits():
    u = W.uniform01(np.uint64(0), np.arange(3, dtype=np.uint64))
    assert u[0] == (0xE220A8397B1DCDAF >> 11) / 2.0 ** 53
    draws = W.uniform01(np.uint64(7), np.arange(200000, dtype=np.uint64))
    assert draws.min() >= 0.0 and draws.max() < 1.0
    # a uniform sample: mean 1/2 and variance 1/12 within a few standard errors
    assert abs(draws.mean() - 0.5) < 5 * np.sqrt(1 / 12 / draws.size)
    assert abs(draws.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / draws.size)


@pytest.mark.parametrize("name,cfg", [("cartpole", 0), ("quadruped", 1), ("hand", 2), ("humanoid", 3)])
def test_a_shard_of_environments_draws_what_the_whole_batch_draws(name, cfg):
    m = W.model(name)
    q, v = W.initial_state(m, cfg, 12)
    qs, vs = W.initial_state(m, cfg, 5, env0=7)
    assert np.array_equal(qs, q[7:12]) and np.array_equal(vs, v[7:12])
    u = W.actions(m, cfg, 12, 0, 6)
    us = W.actions(m, cfg, 5, 2, 3, env0=7)
    assert np.array_equal(us, u[2:5, 7:12])


def test_configs_draw_independent_streams():
    m = W.model("cartpole")
    a = W.initial_state(m, 0, 64)[0]
    b = W.initial_state(m, 3, 64)[0]
    assert not np.any(a == b)


def test_the_recipe_ranges():
    """Cartpole: qpos and qvel in U(+-0.1), controls in U[-1, 1]; the quadruped: at rest in its
    standing pose, controls within 0.3 of the standing targets; the hand: controls in each
    joint's control range."""
    c = W.model("cartpole")
    q, v = W.initial_state(c, 0, 4096)
    assert np.abs(q).max() <= 0.1 and np.abs(v).max() <= 0.1 and np.abs(q).max() > 0.09
    u = W.actions(c, 0, 4096, 0, 4)
    assert u.min() >= -1.0 and u.max() <= 1.0 and u.min() < -0.99 and u.max() > 0.99
    quad = W.model("quadruped")
    q, v = W.initial_state(quad, 1, 16)
    assert np.array_equal(q, np.repeat(quad.qpos_init.astype(np.float32)[None], 16, 0)) and not v.any()
    u = W.actions(quad, 1, 256, 0, 4)
    assert np.abs(u - quad.default_ctrl.astype(np.float32)).max() <= 0.3 + 1e-6
    hand = W.model("hand")
    u = W.actions(hand, 2, 256, 0, 4)
    lo, hi = hand.act_ctrlrange[:, 0].astype(np.float32), hand.act_ctrlrange[:, 1].astype(np.float32)
    assert np.all(u >= lo) and np.all(u <= hi)
