"""Pins for the relaxed (raw-probabilities) oracle, Eqs. 5-10, and its gradient.

  * from a discrete grid, one relaxed step equals the exact expectation of the
    discrete step: the per-cell marginals of the brute-force law (3x3) and the
    Monte-Carlo frequencies of the C oracle (5x5, 4 sigma);
  * p_un + p_burn + p_bd = 1, all in [0, 1], p_un never rises, p_bd never falls;
  * a full tanker mask on a burning cell moves all its mass to burned and stops
    its spread in that step; mask 0 reproduces Eqs. 5-10 unchanged;
  * the autograd gradient of a smooth rollout loss (a random linear functional
    of both planes plus the pooled squared error of Section 4) with respect to
    every parameter and to the initial burning map matches FP64 central finite
    differences (one-sided at mu_den = -1, the edge of the parameter domain).
    PyTorch's binary cross-entropy is left out of this pin: its backward clamps
    the denominator p(1-p) at 1e-12, so it is not the exact derivative for
    cells the fire reaches with probability below 1e-12.
"""
import math

import numpy as np
import pytest
import torch

from oracle import discrete, prob, relaxed
from tests.test_oracle_discrete import _brute_force_law

f64 = torch.float64


def _from_discrete(F):
    F = torch.as_tensor(F)
    p_un = ((F == 0) | (F == 1)).to(f64)
    p_burn = (F == 2).to(f64)
    return p_un, p_burn


def test_relaxed_is_expectation_brute_force():
    F = np.array([[2, 1, 1], [1, 2, 0], [3, 1, 1]], np.uint8)
    rng = np.random.default_rng(4)
    r = rng.uniform(0.1, 2.0, size=(3, 3, 8))
    q = -np.expm1(-r)
    p_c = 0.6
    law = _brute_force_law(F, q, p_c)     # exact law (float64 probabilities)
    m_burn = np.zeros((3, 3))
    m_un = np.zeros((3, 3))
    for k, p in law.items():
        G = np.frombuffer(k, np.uint8).reshape(3, 3)
        m_burn += p * (G == 2)
        m_un += p * ((G == 0) | (G == 1))
    p_un, p_burn = _from_discrete(F)
    # no-fuel cells have zero susceptibility (q = 0 into them)
    rr = torch.as_tensor(r)
    rr[1, 2] = 0.0
    pu, pb = relaxed.relaxed_step(p_un[None], p_burn[None], rr[None], p_c)
    np.testing.assert_allclose(pb[0].numpy(), m_burn, rtol=0, atol=1e-13)
    np.testing.assert_allclose(pu[0].numpy(), m_un, rtol=0, atol=1e-13)


def test_relaxed_is_expectation_monte_carlo():
    rng = np.random.default_rng(12)
    H = W = 5
    F = rng.integers(1, 3, size=(H, W)).astype(np.uint8)
    F[0, 0] = 0
    F[4, 4] = 3
    r = rng.uniform(0.05, 1.0, size=(H, W, 8))
    r[0, 0] = 0.0
    q32 = (-np.expm1(-r)).astype(np.float32)
    r = -np.log1p(-q32.astype(np.float64))   # rates of the float thresholds actually drawn
    p_c = 0.45
    n = 1_000_000
    out = discrete.mc_outcomes(F, q32, p_c, n, seed=5)
    p_un, p_burn = _from_discrete(F)
    pu, pb = relaxed.relaxed_step(p_un[None], p_burn[None], torch.as_tensor(r)[None], p_c)
    fb = (out == 2).mean(axis=0)
    fu = ((out == 0) | (out == 1)).mean(axis=0)
    for f, p in ((fb, pb[0].numpy()), (fu, pu[0].numpy())):
        sigma = np.sqrt(np.maximum(p * (1 - p), 1e-12) / n)
        assert (np.abs(f - p) <= 4 * sigma + 1e-6).all()


def test_conservation_and_monotonicity():
    rng = np.random.default_rng(0)
    N, H, W = 3, 16, 20
    r = torch.as_tensor(rng.uniform(0, 1.5, size=(N, H, W, 8)))
    p_burn = torch.as_tensor((rng.random((N, H, W)) < 0.05).astype(np.float64))
    p_un = 1.0 - p_burn
    pbd = torch.zeros_like(p_un)
    for t in range(60):
        m = torch.as_tensor((rng.random((N, H, W)) < 0.02).astype(np.float64)) * rng.random()
        pu2, pb2 = relaxed.relaxed_step(p_un, p_burn, r, 0.55, m)
        pbd2 = 1.0 - pu2 - pb2
        assert (pu2 <= p_un + 1e-15).all()
        assert (pbd2 >= pbd - 1e-15).all()
        for a in (pu2, pb2, pbd2):
            assert (a >= -1e-15).all() and (a <= 1 + 1e-15).all()
        p_un, p_burn, pbd = pu2, pb2, pbd2


def test_mask_semantics():
    H = W = 5
    r = torch.full((1, H, W, 8), 3.0, dtype=f64)
    p_burn = torch.zeros(1, H, W, dtype=f64)
    p_burn[0, 2, 2] = 1.0
    p_un = 1.0 - p_burn
    m = torch.zeros(1, H, W, dtype=f64)
    m[0, 2, 2] = 1.0
    pu, pb = relaxed.relaxed_step(p_un, p_burn, r, 0.9, m)
    assert (pb == 0).all() and (pu == p_un).all()
    pu0, pb0 = relaxed.relaxed_step(p_un, p_burn, r, 0.9, torch.zeros_like(m))
    pu1, pb1 = relaxed.relaxed_step(p_un, p_burn, r, 0.9, None)
    assert torch.equal(pu0, pu1) and torch.equal(pb0, pb1)


def _param_loss(theta: dict, scn: dict, T: int):
    r = prob.rates(scn["cls"], scn["dem"], scn["V"], scn["Th"], theta["p_base"], theta["alpha_w1"],
                   theta["alpha_w2"], theta["alpha_s"], theta["alpha_gamma"], theta["mu_veg"],
                   theta["mu_den"], 30.0)
    ign = theta["ign"]
    fuel = scn["fuel"]
    p_burn = ign * fuel
    p_un = fuel * (1.0 - ign) + (1.0 - fuel)
    pu, pb = relaxed.relaxed_rollout(p_un, p_burn, r, theta["p_c"], T)
    # smooth loss: random linear functional of both planes + pooled squared error
    lin = (scn["w_un"] * pu).sum() + (scn["w_burn"] * pb).sum()
    mse = ((relaxed.avg_pool(1.0 - pu, 4) - relaxed.avg_pool(scn["target"], 4)) ** 2).mean()
    return lin + mse


def test_autograd_matches_central_differences():
    rng = np.random.default_rng(21)
    N, H, W, C, T = 2, 12, 12, 5, 8
    cls = torch.as_tensor(rng.integers(0, C, size=(N, H, W)))
    mu_den = torch.tensor([0.3, 0.1, -0.2, 0.5, -1.0], dtype=f64)
    scn = dict(cls=cls, dem=torch.as_tensor(rng.random((N, H, W)) * 200.0),
               V=torch.as_tensor(rng.uniform(0, 10, N)), Th=torch.as_tensor(rng.uniform(0, 6.28, N)),
               fuel=(mu_den[cls] > -1).to(f64))
    ign = torch.zeros(N, H, W, dtype=f64)
    ign[:, 6, 6] = 1.0
    ign[1, 3, 8] = 0.7
    # target: the fire map of a rollout with perturbed ("hidden") parameters
    hidden = dict(p_base=torch.tensor(0.7, dtype=f64), alpha_w1=torch.tensor(0.03, dtype=f64),
                  alpha_w2=torch.tensor(0.16, dtype=f64), alpha_s=torch.tensor(0.06, dtype=f64),
                  alpha_gamma=torch.tensor(1.0, dtype=f64), p_c=torch.tensor(0.6, dtype=f64),
                  mu_veg=torch.tensor([0.3, 0.25, 0.1, -0.2, 0.0], dtype=f64), mu_den=mu_den.clone(),
                  ign=ign)
    r_h = prob.rates(cls, scn["dem"], scn["V"], scn["Th"], hidden["p_base"], hidden["alpha_w1"],
                     hidden["alpha_w2"], hidden["alpha_s"], hidden["alpha_gamma"], hidden["mu_veg"],
                     hidden["mu_den"], 30.0)
    pu_h, _ = relaxed.relaxed_rollout(scn["fuel"] * (1 - ign) + (1 - scn["fuel"]), ign * scn["fuel"],
                                      r_h, hidden["p_c"], T)
    scn["target"] = (1.0 - pu_h).detach()
    scn["w_un"] = torch.as_tensor(rng.standard_normal((N, H, W)))
    scn["w_burn"] = torch.as_tensor(rng.standard_normal((N, H, W)))
    theta = dict(p_base=torch.tensor(0.58, dtype=f64), alpha_w1=torch.tensor(0.045, dtype=f64),
                 alpha_w2=torch.tensor(0.131, dtype=f64), alpha_s=torch.tensor(0.078, dtype=f64),
                 alpha_gamma=torch.tensor(1.0, dtype=f64), p_c=torch.tensor(0.5, dtype=f64),
                 mu_veg=torch.tensor([0.4, 0.2, 0.0, -0.3, 0.0], dtype=f64), mu_den=mu_den.clone(),
                 ign=ign)
    for v in theta.values():
        v.requires_grad_(True)
    loss = _param_loss(theta, scn, T)
    grads = torch.autograd.grad(loss, list(theta.values()))
    g = dict(zip(theta.keys(), grads))

    def fd(name, idx=None, h=1e-6):
        def at(delta):
            th = {k: v.detach().clone() for k, v in theta.items()}
            if idx is None:
                th[name] = th[name] + delta
            else:
                th[name][idx] += delta
            return _param_loss(th, scn, T).item()
        return (at(h) - at(-h)) / (2 * h)

    for name in ["p_base", "alpha_w1", "alpha_w2", "alpha_s", "alpha_gamma", "p_c"]:
        assert g[name].item() == pytest.approx(fd(name), rel=1e-6, abs=1e-10), name
    for k in range(C):
        assert g["mu_veg"][k].item() == pytest.approx(fd("mu_veg", k), rel=1e-6, abs=1e-10)
        if mu_den[k] > -1:
            assert g["mu_den"][k].item() == pytest.approx(fd("mu_den", k), rel=1e-6, abs=1e-10)
        else:
            # mu_den = -1 (no fuel) is the edge of the parameter domain: one-sided
            # difference into the domain, looser because of the curvature there
            h = 1e-7
            th = {kk: v.detach().clone() for kk, v in theta.items()}
            base = _param_loss(th, scn, T).item()
            th["mu_den"][k] += h
            one_sided = (_param_loss(th, scn, T).item() - base) / h
            assert g["mu_den"][k].item() == pytest.approx(one_sided, rel=1e-4, abs=1e-9)
    for idx in [(0, 6, 6), (1, 3, 8), (0, 2, 2)]:
        assert g["ign"][idx].item() == pytest.approx(fd("ign", idx), rel=1e-6, abs=1e-10)
