"""Pins for the FP64 rate/threshold oracle (Eqs. 1-4).

Each test fixes something the paper states, chosen so that a plausible slip
(wrong direction angle or row orientation, source and target fields swapped,
slope sign or diagonal distance, radians for degrees, wrap-around at the
border) fails one of them:
  * no wind and flat terrain: all eight directions equal (isotropy);
  * flat terrain: the slope coefficient has no effect;
  * wind toward east (Theta = 0) makes the eastward spread (d = 0) the fastest,
    toward north (Theta = pi/2) the northward one (row - 1), and the ratios
    between directions follow exp(alpha_w2 V (cos(phi_d - Theta) - cos(phi_d' - Theta)));
  * a planar ramp gives the analytic slope angle per direction (in degrees,
    over the diagonal distance for diagonals), and uphill spread is faster;
  * rotating the inputs by 90 degrees and Theta by pi/2 permutes directions;
  * the wind and fuel of Eq. 3 are the source's, the susceptibility the
    target's; a no-fuel target or source gives rate 0;
  * sources outside the grid contribute nothing (no wrap-around).
"""
import math

import numpy as np
import pytest
import torch

from oracle import prob

P = dict(p_base=0.58, alpha_w1=0.045, alpha_w2=0.131, alpha_s=0.078, alpha_gamma=1.0)
MU_VEG = torch.tensor([0.4, 0.2, 0.0, -0.3, 0.0], dtype=torch.float64)
MU_DEN = torch.tensor([0.3, 0.1, -0.2, -0.2, -1.0], dtype=torch.float64)  # class 4: no fuel


def rates(cls, dem, V, Th, **over):
    p = dict(P, **over)
    cls = torch.as_tensor(np.asarray(cls)).long()
    if cls.dim() == 2:
        cls = cls[None]
    dem = torch.as_tensor(np.asarray(dem, np.float64))
    if dem.dim() == 2:
        dem = dem[None]
    V = torch.as_tensor(np.asarray(V, np.float64)).reshape(-1) if np.ndim(V) == 0 else torch.as_tensor(np.asarray(V, np.float64))
    Th = torch.as_tensor(np.asarray(Th, np.float64)).reshape(-1) if np.ndim(Th) == 0 else torch.as_tensor(np.asarray(Th, np.float64))
    return prob.rates(cls, dem, V, Th, p["p_base"], p["alpha_w1"], p["alpha_w2"], p["alpha_s"],
                      p["alpha_gamma"], MU_VEG, MU_DEN, 30.0)[0].numpy()


def test_isotropic_without_wind_and_slope():
    r = rates(np.zeros((9, 9)), np.zeros((9, 9)), 0.0, 1.3)
    inner = r[1:-1, 1:-1]
    assert np.allclose(inner, inner[..., :1], rtol=1e-15, atol=0)
    assert (inner > 0).all()


def test_flat_terrain_slope_coefficient_inert():
    cls = np.random.default_rng(0).integers(0, 4, size=(10, 11))
    a = rates(cls, np.full((10, 11), 321.0), 4.0, 2.0)
    b = rates(cls, np.full((10, 11), 321.0), 4.0, 2.0, alpha_s=0.0)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("theta,expect_d", [(0.0, 0), (math.pi / 2, 2), (math.pi, 4), (3 * math.pi / 2, 6),
                                            (math.pi / 4, 1)])
def test_wind_direction_orientation(theta, expect_d):
    # one burning source at the centre of a 5x5 grid: the target that the wind
    # pushes toward receives the largest rate from it
    r = rates(np.zeros((5, 5)), np.zeros((5, 5)), 8.0, theta)
    dx = prob.DX
    dr = prob.DR
    got = [r[2 + dr[d], 2 + dx[d], d] for d in range(8)]   # target = centre + Delta_d
    assert int(np.argmax(got)) == expect_d
    # the north neighbour is the row above
    if expect_d == 2:
        assert got[2] == r[1, 2, 2]


def test_wind_ratio_closed_form():
    V, Th = 6.5, 0.7
    r = rates(np.zeros((5, 5)), np.zeros((5, 5)), V, Th)[2, 2]
    for d in range(8):
        for e in range(8):
            want = math.exp(P["alpha_w2"] * V * (math.cos(d * math.pi / 4 - Th) - math.cos(e * math.pi / 4 - Th)))
            assert r[d] / r[e] == pytest.approx(want, rel=1e-13)
    # speed factor exp(alpha_w1 V) at the wind's own direction
    r0 = rates(np.zeros((5, 5)), np.zeros((5, 5)), 0.0, Th)[2, 2, 0]
    rw = rates(np.zeros((5, 5)), np.zeros((5, 5)), V, 0.0)[2, 2, 0]
    assert rw / r0 == pytest.approx(math.exp(P["alpha_w1"] * V), rel=1e-13)


def test_ramp_slope_closed_form_and_uphill():
    g = 0.3                                    # rise per metre eastward
    H, W = 6, 7
    dem = np.tile(np.arange(W, dtype=np.float64) * 30.0 * g, (H, 1))
    S = prob.slope_degrees(torch.as_tensor(dem), 30.0).numpy()
    s_e = math.degrees(math.atan(g))
    s_ne = math.degrees(math.atan(g / math.sqrt(2.0)))
    u = (3, 3)
    want = [s_e, s_ne, 0.0, -s_ne, -s_e, -s_ne, 0.0, s_ne]
    np.testing.assert_allclose(S[u], want, rtol=1e-13, atol=1e-12)
    # uphill eastward spread is faster than downhill westward spread
    r = rates(np.zeros((H, W)), dem, 0.0, 0.0)
    assert r[3, 4, 0] > r[3, 2, 4]
    assert r[3, 4, 0] / r[3, 2, 4] == pytest.approx(math.exp(2 * P["alpha_s"] * s_e), rel=1e-12)


def test_rotation_equivariance():
    rng = np.random.default_rng(3)
    cls = rng.integers(0, 5, size=(8, 8))
    dem = rng.random((8, 8)) * 500.0
    V, Th = 5.0, 0.9
    r = rates(cls, dem, V, Th)
    rr = rates(np.rot90(cls).copy(), np.rot90(dem).copy(), V, Th + math.pi / 2)
    # np.rot90 turns the array 90 degrees counter-clockwise; direction d -> d + 2
    for d in range(8):
        np.testing.assert_allclose(np.rot90(r[..., d]), rr[..., (d + 2) % 8], rtol=1e-12, atol=1e-300)


def test_source_wind_and_target_susceptibility():
    H = W = 5
    cls = np.zeros((H, W), np.int64)
    V = np.zeros((1, H, W))
    Th = np.zeros((1, H, W))
    V[0, 2, 2] = 7.0                            # only the centre has wind, blowing east
    r = rates(cls, np.zeros((H, W)), V, Th)
    base = rates(cls, np.zeros((H, W)), 0.0, 0.0)
    for d in range(8):
        ty, tx = 2 + prob.DR[d], 2 + prob.DX[d]  # target fed by the centre in direction d
        want = math.exp(P["alpha_w1"] * 7 + P["alpha_w2"] * 7 * (math.cos(d * math.pi / 4) - 1))
        assert r[ty, tx, d] / base[ty, tx, d] == pytest.approx(want, rel=1e-13)
    # the centre as a target (fed by windless sources) is unaffected
    np.testing.assert_allclose(r[2, 2], base[2, 2], rtol=1e-15)
    # a no-fuel target has zero susceptibility; a no-fuel source has zero potential
    cls2 = cls.copy()
    cls2[2, 2] = 4
    r2 = rates(cls2, np.zeros((H, W)), 0.0, 0.0)
    assert (r2[2, 2] == 0).all()
    for d in range(8):
        assert r2[2 + prob.DR[d], 2 + prob.DX[d], d] == 0
        assert r2[2 + prob.DR[d], 2 + prob.DX[d], (d + 1) % 8] > 0
    # fuel modifiers enter twice (source and target) when both cells share a class
    cls3 = np.full((H, W), 1)
    r3 = rates(cls3, np.zeros((H, W)), 0.0, 0.0)
    f = (1 + 0.2) * (1 + 0.1)
    assert r3[2, 2, 0] == pytest.approx(P["alpha_gamma"] * P["p_base"] * f * f, rel=1e-14)


def test_border_sources_absent():
    r = rates(np.zeros((4, 6)), np.zeros((4, 6)), 3.0, 1.0)
    # column 0 has no western sources (directions whose source is at x - 1)
    for d in range(8):
        if prob.DX[d] == 1:
            assert (r[:, 0, d] == 0).all()
        if prob.DX[d] == -1:
            assert (r[:, -1, d] == 0).all()
        if prob.DR[d] == 1:      # source at row - 1
            assert (r[0, :, d] == 0).all()
        if prob.DR[d] == -1:
            assert (r[-1, :, d] == 0).all()
    assert (r[1:-1, 1:-1] > 0).all()


def test_threshold_is_poisson_complement():
    r = torch.tensor([0.0, 1e-12, 0.3, 5.0, 60.0], dtype=torch.float64)
    q = prob.thresholds(r).numpy()
    assert q[0] == 0.0 and q[-1] == 1.0
    assert q[1] == pytest.approx(1e-12, rel=1e-9)
    assert q[2] == pytest.approx(1 - math.exp(-0.3), rel=1e-15)
