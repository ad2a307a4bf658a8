"""Batched RL rollouts: ragged batches in size classes (one persistent launch
per class, side by side on forked streams), auto-reset, CUDA-graph capture and
the autotuner.

  * a graph-captured 60-step rollout (one jwf_step per step plus the reward)
    replays bit-identically to the same launches issued eagerly;
  * the graph rollout of a ragged batch with auto-reset and an episode limit
    equals the oracle's rollout step by step (states, counts, done flags,
    step counters and episode numbers; a restarted env draws the fresh
    stream of episode + 1);
  * rewards follow Section 4 (penalty per burning cell, +10 on extinction);
  * autotuned block sizes and round lengths leave every result unchanged.
"""
import numpy as np
import pytest
import torch

from oracle import discrete
from paper_2512_06102_gb300 import autotune, jwf, rollout, scenarios
from tests.gpu_util import make_sim, oracle_tables, require_gpu, to

pytestmark = pytest.mark.gpu


def _ragged(n, seed, lo=32, hi=512):
    sides = scenarios.ragged_sides(n, lo, hi, seed=seed)
    return scenarios.make_scenario(sides, np.roll(sides, 1), seed=seed)


def test_size_classes_present():
    require_gpu()
    scn = _ragged(40, 1)
    sim = make_sim(scn)
    cl = sim.size_classes()
    assert len(cl) >= 3 and cl == sorted(cl, reverse=True)
    sim.close()


def test_graph_equals_eager_fused_auto_reset():
    require_gpu()
    scn = _ragged(24, 2)
    T = 60
    drops = to(scenarios.drops(T, scn.H, scn.W, seed=2))
    res = []
    for capture in (True, False):
        sim = make_sim(scn, seed=4, t_max=25, auto_reset=True)
        sim.set_kernel(jwf.KERNEL_FUSED)
        sim.set_terrain(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
        sim.load_state(to(scn.F0))
        ro = rollout.GraphRollout(sim, T, drops, capture=capture, steps_per_launch=1 if capture else 7)
        sim.load_state(to(scn.F0))
        r = ro.run().clone()
        torch.cuda.synchronize()
        s, t, ep = (x.cpu().numpy().copy() for x in sim.state_views())
        res.append((s, t, ep, r.cpu().numpy(), ro.burning.cpu().numpy(), ro.burnt.cpu().numpy(),
                    ro.done.cpu().numpy()))
        sim.close()
    for a, b in zip(*res):
        np.testing.assert_array_equal(a, b)
    assert (res[0][2] >= 2).all()                       # envs restarted


def test_graph_rollout_matches_oracle():
    require_gpu()
    scn = _ragged(10, 3, 32, 300)
    q32 = oracle_tables(scn)[0]
    T = 45
    drops_np = scenarios.drops(T, scn.H, scn.W, seed=3)
    sim = make_sim(scn, seed=6, t_max=20, auto_reset=True)
    sim.set_kernel(jwf.KERNEL_RESIDENT)
    sim.set_probs(to(q32))
    sim.load_state(to(scn.F0))
    ro = rollout.GraphRollout(sim, T, to(drops_np))
    sim.load_state(to(scn.F0))
    rew = ro.run().cpu().numpy()
    torch.cuda.synchronize()
    orc = discrete.Rollout(scn.H, scn.W, scn.F0, q32, scn.params.p_continue, seed=6, t_max=20, auto_reset=True)
    ob, od, odone = orc.step(T, drops_np)
    np.testing.assert_array_equal(ro.burning.cpu().numpy(), ob)
    np.testing.assert_array_equal(ro.burnt.cpu().numpy(), od)
    np.testing.assert_array_equal(ro.done.cpu().numpy(), odone)
    s, t, ep = (x.cpu().numpy() for x in sim.state_views())
    np.testing.assert_array_equal(s, orc.F)
    np.testing.assert_array_equal(t, orc.t)
    np.testing.assert_array_equal(ep, orc.episode)
    # Section 4 reward from the oracle's counts
    prev = np.vstack([np.zeros((1, scn.N), np.int32), ob[:-1]])
    want = -0.01 * ob + 10.0 * ((ob == 0) & (prev > 0))
    np.testing.assert_allclose(rew, want.astype(np.float32), rtol=0, atol=1e-6)
    sim.close()


@pytest.mark.parametrize("kernel", [jwf.KERNEL_FUSED, jwf.KERNEL_TILED_FUSED])
def test_autotune_keeps_results(kernel, tmp_path, monkeypatch):
    require_gpu()
    monkeypatch.setenv("JWF_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    scn = _ragged(16, 5) if kernel == jwf.KERNEL_FUSED else scenarios.make_scenario(700, 600, N=2, seed=5)
    k = 40
    drops = to(scenarios.drops(k, scn.H, scn.W, seed=5))
    terrain = (to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    F0 = to(scn.F0)
    outs = []
    for tuned in (False, True):
        sim = make_sim(scn, seed=7)
        sim.set_kernel(kernel)
        sim.set_terrain(*terrain)
        if tuned:
            choice = autotune.tune(sim, F0, drops, kernel=kernel, probe_steps=16)
            assert choice
            again = autotune.tune(sim, F0, drops, kernel=kernel, probe_steps=16)     # from the cache
            assert again == choice
            kk = autotune.tune_steps_per_launch(sim, F0, drops, k)
            assert 1 <= kk <= k
        sim.load_state(F0)
        o = [x.cpu().numpy() for x in sim.step(k, drops)]
        outs.append((sim.state().cpu().numpy(), o))
        sim.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    for a, b in zip(outs[0][1], outs[1][1]):
        np.testing.assert_array_equal(a, b)
