"""The fused step kernels' two-level ignition test (Section 3 "Stochastic
update", Eqs. 1-4): a pair's draw u is compared with a plain-float
probability p_f when it lies farther than a bound B from it, and with the
double-float probability p otherwise, so the outcome must always be u < p.
That holds when |p_f - p| <= B; B is four times the sum of the steps' error
bounds, so the test asks for |p_f - p| <= B / 4 on adversarial tuples: every
class pair, slopes from flat to nearly vertical, equal elevations, and wind
and slope parts of the exponent far outside the benchmark's range, under
several parameter sets.  It also checks that the exact path is rare (the
draws within B of p_f are a small fraction).
"""
import numpy as np
import pytest
import torch

from paper_2512_06102_gb300 import jwf, scenarios
from tests.gpu_util import require_gpu, to

pytestmark = pytest.mark.gpu

N = 1 << 22


def _tuples(rng, n, n_classes, wide):
    cv = rng.integers(0, n_classes, n).astype(np.uint8)
    cu = rng.integers(0, n_classes, n).astype(np.uint8)
    zv = rng.uniform(0.0, 2000.0, n).astype(np.float32)
    kind = rng.integers(0, 4, n)
    dz = np.where(kind == 0, rng.uniform(-2000.0, 2000.0, n),          # any slope up to ~89 degrees
         np.where(kind == 1, rng.uniform(-5.0, 5.0, n),                # gentle
         np.where(kind == 2, 0.0, rng.uniform(-60.0, 60.0, n))))       # flat; about one cell size
    zu = (zv - dz).astype(np.float32)
    d = rng.integers(0, 8, n).astype(np.int32)
    lim = 20.0 if wide else 3.0
    w = rng.uniform(-lim, lim, n)
    hi = w.astype(np.float32)
    lo = (w - hi.astype(np.float64)).astype(np.float32)
    return cv, cu, zv, zu, np.stack([hi, lo], 1), d


@pytest.mark.parametrize("case, params", list(enumerate([
    {},                                                          # the benchmark's coefficients
    {"alpha_w1": 0.2, "alpha_w2": 0.5},                          # strong wind
    {"alpha_s": 0.5, "p_base": 2.0},                             # a large slope coefficient, high base rate
    {"alpha_s": -0.2, "p_base": 0.05},                           # negative slope effect, low base rate
])))
def test_fast_probability_bound_holds(case, params):
    require_gpu()
    scn = scenarios.make_scenario(32, 32, N=1, seed=0)
    P = jwf.ParamSet.from_any(scn.params)
    for k, v in params.items():
        setattr(P, k, v)
    n_classes = len(P.mu_veg)
    sim = jwf.Sim([32], [32], n_classes=n_classes, seed=0)
    sim.set_params(P)
    rng = np.random.default_rng(100 + case)
    for wide in (False, True):
        cv, cu, zv, zu, wx, d = (to(a) for a in _tuples(rng, N, n_classes, wide))
        out = sim.check_prob_bound(cv, cu, zv, zu, wx.reshape(-1), d)
        torch.cuda.synchronize()
        pf, B, p = out[:, 0].double(), out[:, 1].double(), out[:, 2].double()
        fin = torch.isfinite(p)
        assert fin.float().mean() > 0.99
        ratio = ((pf - p).abs() / B)[fin]
        assert float(ratio.max()) <= 0.25, f"max |p_f - p| / B = {float(ratio.max()):.3f}"
        # the exact path runs for draws within B of p_f
        assert float((2 * B[fin]).clamp(max=1).mean()) < 1e-3
        assert ((p > 0) & (p < 1)).float().mean() > 0.2          # the tuples span the probability range
    sim.close()
