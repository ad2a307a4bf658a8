"""The air-tanker agent environment (Section 4) on the GPU against its oracle.

With the oracle's FP32 table and the same seed, every step's observation,
reward, done flag, agent state and grid state equal the oracle's, over
episodes that restart (auto-reset, random agent position and ignition), for
random actions, on 20 x 20 grids (one warp per grid, and the three-launch
path) and on 40 x 36 grids; the fused kernel (rates from the terrain) gives
the same trajectory as the table kernel; a CUDA-graph rollout gives the same
rewards as eager steps.
"""
import numpy as np
import pytest
import torch

from oracle import agent as oagent
from paper_2512_06102_gb300 import jwf, scenarios, tanker
from tests.gpu_util import make_sim, oracle_tables, require_gpu, to

pytestmark = pytest.mark.gpu

N, S, T = 48, 20, 150


def _fire_free(scn):
    F0 = scn.F0.copy()
    F0[F0 == 2] = 1
    return F0


def _gpu_env(scn, F0, kernel, q=None, seed=17):
    sim = make_sim(scn, seed=seed, auto_reset=True, t_max=60)
    if q is None:
        sim.set_terrain(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    else:
        sim.set_probs(to(q))
    sim.set_kernel(kernel)
    return sim, tanker.TankerEnv(sim, to(F0), water0=6, obs_k=5, burn_penalty=0.02, random_fire=True)


@pytest.mark.parametrize("shape,kernel", [((S, S), jwf.KERNEL_RESIDENT),     # one warp per grid
                                          ((S, S), jwf.KERNEL_PLAIN),        # act + step + post launches
                                          ((40, 36), jwf.KERNEL_RESIDENT)])  # larger than a warp's grid
def test_tanker_matches_oracle(shape, kernel):
    require_gpu()
    scn = scenarios.make_scenario(shape[0], shape[1], N=N, seed=51)
    F0 = _fire_free(scn)
    q32 = oracle_tables(scn)[0]
    sim, env = _gpu_env(scn, F0, kernel, q32)
    ora = oagent.TankerOracle(scn.H, scn.W, F0, q32, scn.params.p_continue, seed=17, t_max=60, water0=6, obs_k=5,
                              burn_penalty=0.02, random_fire=True)
    np.testing.assert_array_equal(env.reset().cpu().numpy(), ora.reset())
    np.testing.assert_array_equal(env.agent.cpu().numpy(), ora.agent)
    rng = np.random.default_rng(3)
    restarts = 0
    for t in range(T):
        a = rng.integers(0, 10, size=N).astype(np.int32)
        obs, rew, done = env.step(to(a))
        o_obs, o_rew, o_done = ora.step(a)
        np.testing.assert_array_equal(done.cpu().numpy(), o_done)
        np.testing.assert_array_equal(rew.cpu().numpy(), o_rew)
        np.testing.assert_array_equal(env.agent.cpu().numpy(), ora.agent)
        np.testing.assert_array_equal(obs.cpu().numpy(), o_obs)
        np.testing.assert_array_equal(sim.state().cpu().numpy(), ora.ro.F)
        restarts += int(o_done.sum())
    sim.close()
    assert restarts > N          # several episodes per grid, extinctions included


def test_fused_and_graph_rollouts():
    require_gpu()
    scn = scenarios.make_scenario(S, S, N=N, seed=52)
    F0 = _fire_free(scn)
    acts = to(np.random.default_rng(4).integers(0, 10, size=(T, N)).astype(np.int32))
    out = {}
    for kernel in (jwf.KERNEL_RESIDENT, jwf.KERNEL_FUSED):
        sim, env = _gpu_env(scn, F0, kernel)
        if kernel == jwf.KERNEL_RESIDENT:
            sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
        env.reset()
        r = torch.stack([env.step(acts[t])[1].clone() for t in range(T)])
        out[kernel] = (r.cpu().numpy(), sim.state().cpu().numpy())
        if kernel == jwf.KERNEL_FUSED:
            # the same rollout as one graph (the capture's warm-up step is replayed from a reset)
            env.reset()
            g = tanker.GraphTankerRollout(env, acts)
            env.reset()
            rg = g.run().clone()
            torch.cuda.synchronize()
            out["graph"] = (rg.cpu().numpy(), sim.state().cpu().numpy())
        sim.close()
    np.testing.assert_array_equal(out[jwf.KERNEL_RESIDENT][0], out[jwf.KERNEL_FUSED][0])
    np.testing.assert_array_equal(out[jwf.KERNEL_RESIDENT][1], out[jwf.KERNEL_FUSED][1])
    np.testing.assert_array_equal(out["graph"][0], out[jwf.KERNEL_FUSED][0])
    np.testing.assert_array_equal(out["graph"][1], out[jwf.KERNEL_FUSED][1])
