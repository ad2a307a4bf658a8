"""The resident kernels' work-queue order changes no result: a ragged batch
(several size classes) stepped in the default, ascending-index and random
priority orders (jwf_set_env_priority), and with the launch split after 8
steps and the second part reordered by burning count on the device
(jwf_set_reorder_steps), gives the oracle's final states (table variant, the
oracle's FP32 table) and the same per-step counts and done flags, bit for
bit, for both resident variants."""
import numpy as np
import pytest

from oracle import discrete
from paper_2512_06102_gb300 import jwf, scenarios
from tests.gpu_util import make_sim, oracle_tables, require_gpu, to

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kernel", [jwf.KERNEL_RESIDENT, jwf.KERNEL_FUSED])
def test_priority_order_changes_nothing(kernel):
    require_gpu()
    k = 30
    rng = np.random.default_rng(5)
    H = rng.integers(20, 150, size=12)
    W = rng.integers(20, 150, size=12)
    scn = scenarios.make_scenario(H, W, seed=71)
    drops = scenarios.drops(k, scn.H, scn.W, seed=7)
    q32 = oracle_tables(scn)[0]
    ro = discrete.Rollout(scn.H, scn.W, scn.F0, q32, scn.params.p_continue, seed=3)
    ro.step(k, np.ascontiguousarray(drops))
    N = len(scn.H)
    base = None
    prios = (None, np.arange(N, dtype=np.float32), rng.random(N).astype(np.float32))
    for prio, split in [(p, 0) for p in prios] + [(None, 8), (prios[2], 5)]:
        sim = make_sim(scn, seed=3)
        sim.set_reorder_steps(split)
        if kernel == jwf.KERNEL_RESIDENT:
            sim.set_probs(to(q32))
        else:
            sim.set_terrain(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
        sim.set_kernel(kernel)
        sim.set_env_priority(prio)
        sim.load_state(to(scn.F0))
        out = [x.cpu().numpy() for x in sim.step(k, to(drops))]
        st = sim.state().cpu().numpy()
        sim.close()
        if kernel == jwf.KERNEL_RESIDENT:
            np.testing.assert_array_equal(st, ro.F)
        if base is None:
            base = (st, *out)
        else:
            for x, y in zip((st, *out), base):
                np.testing.assert_array_equal(x, y)
