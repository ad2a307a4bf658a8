"""Step kernels whose block-wide work queue overflows (Section 3 "Stochastic
update", Eq. 4): a fire far larger than the queue's capacity (1024 work items
an env in the resident step, 4096 a tile in the tiled step).  A warp whose
reservation runs past the capacity voids the slots it got and evaluates its
chunk itself; the outcome must still equal the oracle bit for bit (states,
burning and burned counts, done flags), for every kernel, table and fused.
"""
import numpy as np
import pytest
import torch

from oracle import discrete
from paper_2512_06102_gb300 import jwf, scenarios
from tests.gpu_util import make_sim, oracle_tables, require_gpu, to

pytestmark = pytest.mark.gpu

FUSED = (jwf.KERNEL_FUSED, jwf.KERNEL_TILED_FUSED)


def _big_fire(seed):
    scn = scenarios.make_scenario(192, 256, N=2, seed=seed)
    F0 = scn.F0.reshape(2, 192, 256).copy()
    # a 70 x 100 block of burning cells in each grid (about 7000 remain-burning
    # draws in the first step alone), placed differently in the two grids
    for e, (y0, x0) in enumerate(((40, 60), (100, 130))):
        blk = F0[e, y0:y0 + 70, x0:x0 + 100]
        F0[e, y0:y0 + 70, x0:x0 + 100] = np.where(blk != 0, 2, 0)
    scn.F0 = F0.reshape(-1)
    return scn


def _gpu_table(scn):
    sim = make_sim(scn)
    sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    q = sim.probs()[0].cpu().numpy().copy()
    sim.close()
    return q


@pytest.mark.parametrize("kernel", [jwf.KERNEL_PLAIN, jwf.KERNEL_RESIDENT, jwf.KERNEL_TILED, jwf.KERNEL_FUSED,
                                    jwf.KERNEL_TILED_FUSED])
def test_overflowing_queue_equals_oracle(kernel):
    require_gpu()
    scn = _big_fire(seed=21)
    assert (scn.F0 == 2).sum() > 2 * 5000
    q32 = _gpu_table(scn) if kernel in FUSED else oracle_tables(scn)[0]
    sim = make_sim(scn, seed=9)
    sim.set_kernel(kernel)
    if kernel in FUSED:
        sim.set_terrain(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    else:
        sim.set_probs(to(q32))
    sim.load_state(to(scn.F0))
    outs = [[x.cpu().numpy() for x in sim.step(kk)] for kk in (1, 3, 4)]
    torch.cuda.synchronize()
    sim.sync()
    state = sim.state().cpu().numpy()
    sim.close()
    ro = discrete.Rollout(scn.H, scn.W, scn.F0, q32, scn.params.p_continue, seed=9)
    ob, od, odone = ro.step(8)
    np.testing.assert_array_equal(state, ro.F)
    np.testing.assert_array_equal(np.concatenate([o[0] for o in outs]), ob)
    np.testing.assert_array_equal(np.concatenate([o[1] for o in outs]), od)
    np.testing.assert_array_equal(np.concatenate([o[2] for o in outs]), odone)
    assert ob[0].min() > 2000            # the fires are still large after the first step
