"""The seeded generator: deterministic, shaped like the workloads it stands in for."""
import numpy as np

from paper_2512_06102_gb300 import scenarios as sc


def test_deterministic_and_shaped():
    a = sc.make_scenario(128, 128, N=6, seed=3)
    b = sc.make_scenario(128, 128, N=6, seed=3)
    for k in ("cls", "dem", "wind_speed", "wind_dir", "F0"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))
    assert a.cls.shape == (6 * 128 * 128,) and a.cls.max() < sc.N_CLASSES
    nofuel = (~sc.burnable_classes(a.params.mu_den)[a.cls]).mean()
    assert 0.07 < nofuel < 0.13                  # about 10% non-burnable
    assert a.dem.min() >= 0 and a.dem.max() <= 2000.0 + 1e-3
    assert (a.wind_speed >= 0).all() and (a.wind_speed <= 10).all()
    for e in range(6):
        F = a.env(e, a.F0)
        assert 1 <= (F == 2).sum() <= 3
        assert ((F == 0) == ~sc.burnable_classes(a.params.mu_den)[a.env(e, a.cls)]).all()


def test_ragged_and_drops():
    s = sc.ragged_sides(2000, 32, 512, seed=1)
    assert s.min() >= 32 and s.max() <= 512
    assert 100 < np.median(s) < 160                       # log-uniform median ~ 128
    d = sc.drops(5, [40, 64], [50, 64], seed=2)
    assert d.shape == (5, 2, 2)
    assert (d[:, 0, 0] < 50).all() and (d[:, 0, 1] < 40).all()
