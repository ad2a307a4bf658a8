"""GPU probability kernel (Eqs. 1-4) against the FP64 oracle: 1e-6 relative."""
import numpy as np
import pytest
import torch

from paper_2512_06102_gb300 import scenarios
from tests.gpu_util import make_sim, oracle_tables, require_gpu, to

pytestmark = pytest.mark.gpu
REL = 1e-6


def _check(gpu, ref):
    err = np.abs(gpu.astype(np.float64) - ref)
    bad = err > REL * np.abs(ref)
    assert not bad.any(), f"{bad.sum()} entries off; worst rel {np.max(err / np.maximum(np.abs(ref), 1e-300))}"
    assert np.array_equal(gpu == 0, ref == 0)


@pytest.mark.parametrize("shape", [(128, 128, 8), (37, 45, 3), (1, 17, 2), (130, 1, 2)])
def test_table_matches_fp64(shape):
    require_gpu()
    H, W, N = shape
    scn = scenarios.make_scenario(H, W, N=N, seed=5)
    sim = make_sim(scn, keep_rates=True)
    sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    q, r = (t.cpu().numpy() for t in sim.probs())
    _, _, q64, r64 = oracle_tables(scn)
    _check(q, q64)
    _check(r, r64)


def test_table_ragged_and_per_cell_wind():
    require_gpu()
    from oracle import prob
    sides = scenarios.ragged_sides(6, 32, 200, seed=2)
    scn = scenarios.make_scenario(sides, sides[::-1], seed=3)
    rng = np.random.default_rng(0)
    ws = rng.uniform(0, 10, scn.cls.size).astype(np.float32)
    wd = rng.uniform(0, 2 * np.pi, scn.cls.size).astype(np.float32)
    sim = make_sim(scn, keep_rates=True, wind_per_cell=True)
    sim.precompute_probs(to(scn.cls), to(scn.dem), to(ws), to(wd))
    q, r = (t.cpu().numpy() for t in sim.probs())
    p = scn.params.as_dict()
    for e in range(scn.N):
        o0, o1 = scn.offsets[e], scn.offsets[e + 1]
        Hs, Ws = int(scn.H[e]), int(scn.W[e])
        _, _, q64, r64 = prob.table_f32(scn.env(e, scn.cls)[None], scn.env(e, scn.dem)[None],
                                        ws[o0:o1].reshape(1, Hs, Ws), wd[o0:o1].reshape(1, Hs, Ws), p, 30.0)
        _check(q[o0:o1], q64.reshape(-1, 8))
        _check(r[o0:o1], r64.reshape(-1, 8))


def test_table_full_size_sampled():
    """4096 x 128^2 (the batched workload): oracle on a sample of envs."""
    require_gpu()
    from oracle import prob
    N, H, W = 4096, 128, 128
    scn = scenarios.make_scenario(H, W, N=N, seed=0)
    sim = make_sim(scn)
    sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    q, _ = sim.probs()
    rng = np.random.default_rng(1)
    p = scn.params.as_dict()
    for e in sorted(rng.choice(N, 12, replace=False).tolist()) + [0, N - 1]:
        o0, o1 = scn.offsets[e], scn.offsets[e + 1]
        _, _, q64, _ = prob.table_f32(scn.env(e, scn.cls)[None], scn.env(e, scn.dem)[None],
                                      scn.wind_speed[e:e + 1], scn.wind_dir[e:e + 1], p, 30.0)
        _check(q[o0:o1].cpu().numpy(), q64.reshape(-1, 8))
