"""The kernels the benchmark times, against the oracle directly.

The fused step kernels evaluate the ignition probabilities of Eqs. 1-4 on the
spot (the same rate code as the table kernel).  Here the oracle is handed the
GPU's own float table, read back through jwf_get_probs after
jwf_precompute_probs, and steps with the same Philox stream (Section 3,
"Stochastic update"; Eq. 4 per burning neighbour): states, burning and burned
counts and done flags of the fused kernels must equal it bit for bit, in the
benchmark's own launch configurations:

  * the batched workload, 4096 grids of 128 x 128, one 200-step episode with a
    3 x 3 drop per grid and step, fused resident kernel with the launch split
    after 12 steps (reordered by burning cells), sampled grids, and the same
    episode run twice (every timed episode does the same work);
  * the same episode with a per-step wind series (one table per step);
  * one 4096 x 4096 grid of the large-map workload (8 grids, drops), fused
    tiled kernel, 256 threads a tile and 16 steps a round, 48 steps.
"""
import numpy as np
import pytest
import torch

from oracle import discrete
from paper_2512_06102_gb300 import jwf, scenarios
from tests.gpu_util import make_sim, require_gpu, to

pytestmark = pytest.mark.gpu

N_ENVS, SIDE, EPISODE, REORDER = 4096, 128, 200, 12


def _gpu_table(scn, ws=None, wd=None):
    """The GPU's own q table (float32 [cells, 8]) from jwf_precompute_probs."""
    sim = make_sim(scn)
    sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed if ws is None else ws),
                         to(scn.wind_dir if wd is None else wd))
    q = sim.probs()[0].clone()
    torch.cuda.synchronize()
    sim.close()
    return q


def _rows(q_dev, scn, envs):
    return np.concatenate([q_dev[scn.offsets[e]:scn.offsets[e + 1]].cpu().numpy() for e in envs])


def _fused_episode(scn, drops_d, seed, series=None):
    sim = make_sim(scn, seed=seed)
    sim.set_kernel(jwf.KERNEL_FUSED)
    sim.set_reorder_steps(REORDER)
    sim.load_state(to(scn.F0))
    sim.set_terrain(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    if series is not None:
        sim.set_wind_series(*series)
    out = sim.step(EPISODE, drops_d)
    torch.cuda.synchronize()
    sim.sync()
    res = (sim.state().cpu().numpy(), [x.cpu().numpy() for x in out])
    sim.close()
    return res


def _sample(b, rng, n_random=40):
    """Grids to check against the oracle: the first and last, the longest and
    shortest fires, the largest final fires, and a random draw."""
    N = b.shape[1]
    alive = (b > 0).sum(0)
    pick = {0, N - 1, int(alive.argmax()), int(alive.argmin())}
    pick.update(int(x) for x in np.argsort(-b[REORDER])[:6])       # most burning cells at the split
    pick.update(int(x) for x in np.argsort(-alive)[:6])
    pick.update(int(x) for x in rng.choice(N, n_random, replace=False))
    return sorted(pick)


def _check_against_oracle(scn, drops, seed, state, out, sample, q_rows_per_step):
    """q_rows_per_step(t) -> float32 [cells of the sample, 8] for step t."""
    H = scn.H[sample]
    W = scn.W[sample]
    F0s = np.concatenate([scn.env(e, scn.F0).reshape(-1) for e in sample])
    ro = discrete.Rollout(H, W, F0s, q_rows_per_step(0), scn.params.p_continue, seed=seed,
                          env_ids=np.array(sample, np.int32))
    dr = np.ascontiguousarray(drops[:, sample])
    if getattr(q_rows_per_step, "static", False):
        ob, od, odone = ro.step(EPISODE, dr)
    else:
        parts = []
        for t in range(EPISODE):
            ro.q = np.ascontiguousarray(q_rows_per_step(t), np.float32)
            parts.append(ro.step(1, dr[t:t + 1]))
        ob, od, odone = (np.concatenate([p[i] for p in parts]) for i in range(3))
    for i, e in enumerate(sample):
        np.testing.assert_array_equal(state[scn.offsets[e]:scn.offsets[e + 1]], ro.env_state(i).reshape(-1),
                                      err_msg=f"grid {e}")
    np.testing.assert_array_equal(out[0][:, sample], ob)
    np.testing.assert_array_equal(out[1][:, sample], od)
    np.testing.assert_array_equal(out[2][:, sample], odone)


def test_bench_episode_fused_equals_oracle_on_gpu_table():
    require_gpu()
    scn = scenarios.make_scenario(SIDE, SIDE, N=N_ENVS, seed=0)
    drops = scenarios.drops(EPISODE, scn.H, scn.W, seed=0)
    drops_d = to(drops)
    seed = 1000
    state, out = _fused_episode(scn, drops_d, seed)
    # every timed episode repeats the same work: a second run is identical
    state2, out2 = _fused_episode(scn, drops_d, seed)
    np.testing.assert_array_equal(state, state2)
    for a, b in zip(out, out2):
        np.testing.assert_array_equal(a, b)
    sample = _sample(out[0], np.random.default_rng(5))
    q = _gpu_table(scn)
    rows = _rows(q, scn, sample)
    fn = lambda t: rows
    fn.static = True
    _check_against_oracle(scn, drops, seed, state, out, sample, fn)
    # properties of every grid: no-fuel cells never change; a grid is done
    # exactly when it has no burning cell (no step limit here)
    assert ((state == 0) == (scn.F0 == 0)).all()
    np.testing.assert_array_equal(out[2] == 1, out[0] == 0)
    assert (out[0][-1] > 0).sum() < N_ENVS and (out[1][-1] > 0).all()


def test_bench_wind_series_episode_equals_oracle_on_per_step_gpu_tables():
    require_gpu()
    scn = scenarios.make_scenario(SIDE, SIDE, N=N_ENVS, seed=0)
    drops = scenarios.drops(EPISODE, scn.H, scn.W, seed=0)
    rng = np.random.default_rng(11)
    ws = rng.uniform(0.0, 10.0, size=(EPISODE, N_ENVS)).astype(np.float32)
    wd = rng.uniform(0.0, 2 * np.pi, size=(EPISODE, N_ENVS)).astype(np.float32)
    seed = 1000
    state, out = _fused_episode(scn, to(drops), seed, series=(to(ws), to(wd)))
    sample = _sample(out[0], np.random.default_rng(6), n_random=12)
    # the table of step t from that step's wind row, built by the GPU table
    # kernel when the oracle reaches step t
    sim = make_sim(scn)
    cls, dem = to(scn.cls), to(scn.dem)

    def table(t):
        sim.precompute_probs(cls, dem, to(ws[t]), to(wd[t]))
        return _rows(sim.probs()[0], scn, sample)

    _check_against_oracle(scn, drops, seed, state, out, sample, table)
    sim.close()


def test_large_map_tiled_fused_equals_oracle_on_gpu_table():
    require_gpu()
    N, S, k, e = 8, 4096, 48, 3
    scn = scenarios.make_scenario(S, S, N=N, seed=200)
    drops = scenarios.drops(k, scn.H, scn.W, seed=200)
    sim = make_sim(scn, seed=0)
    sim.set_kernel(jwf.KERNEL_TILED_FUSED, 256)
    sim.set_round_steps(16)
    sim.set_terrain(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    sim.load_state(to(scn.F0))
    out = [x.cpu().numpy() for x in sim.step(k, to(drops))]
    torch.cuda.synchronize()
    sim.sync()
    st = sim.state()[scn.offsets[e]:scn.offsets[e + 1]].cpu().numpy()
    sim.close()
    q = _gpu_table(scn)
    qe = q[scn.offsets[e]:scn.offsets[e + 1]].cpu().numpy()
    del q
    torch.cuda.empty_cache()
    ro = discrete.Rollout([S], [S], scn.env(e, scn.F0).reshape(-1), qe, scn.params.p_continue, seed=0,
                          env_ids=[e])
    ob, od, odone = ro.step(k, np.ascontiguousarray(drops[:, e:e + 1]))
    np.testing.assert_array_equal(st, ro.F)
    np.testing.assert_array_equal(out[0][:, e:e + 1], ob)
    np.testing.assert_array_equal(out[1][:, e:e + 1], od)
    np.testing.assert_array_equal(out[2][:, e:e + 1], odone)
    assert ob[-1, 0] > 0 and od[-1, 0] > od[0, 0]          # a live fire, growing
