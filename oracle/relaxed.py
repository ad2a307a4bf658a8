"""FP64 oracle for the deterministic (raw-probabilities) update of JaxWildfire.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.

Written from arXiv 2512.06102, Section 3, "Deterministic (raw-probabilities)
update", Eqs. 5-10, with p_ignite from Eq. 4.  Plain PyTorch float64 ops, so
that autograd supplies the reference gradient of a rollout (the gradient is
the derivative of this forward; the tests pin it with central differences).

Readings (where the paper is silent):
  * In Eq. 4 the burning indicator b(u) is replaced by p_burn(u), so
    p_ignite(v) = 1 - exp(-sum_d p_burn(v - Delta_d) * r(v, d)).
  * The burned-out probability is implicit: p_bd = 1 - p_un - p_burn.
  * The tanker mask m(v) in [0, 1] acts before the spread, as in the discrete
    step: the burning mass (1 - m) * p_burn is what spreads and continues, and
    m * p_burn goes to burned.  (With m = 0 this is exactly Eqs. 5-10.)
"""
from __future__ import annotations

import torch

from .prob import shift_from_source


def relaxed_step(p_un: torch.Tensor, p_burn: torch.Tensor, r: torch.Tensor,
                 p_continue, mask: torch.Tensor | None = None):
    """One step of Eqs. 5-10.  p_un, p_burn: [N, H, W]; r: [N, H, W, 8]."""
    pb = p_burn if mask is None else (1.0 - mask) * p_burn
    lam = torch.zeros_like(p_un)
    for d in range(8):
        lam = lam + shift_from_source(pb, d, 0.0) * r[..., d]   # gamma(v) * lambda(v)
    p_ignite = -torch.expm1(-lam)                                # Eq. 4
    newly_burning = p_un * p_ignite                              # Eq. 5
    continuing = pb * p_continue                                 # Eq. 6
    p_burn_next = newly_burning + continuing                     # Eq. 8
    p_un_next = p_un - newly_burning                             # Eq. 9
    return p_un_next, p_burn_next                                # Eq. 10 is implicit


def relaxed_rollout(p_un, p_burn, r, p_continue, T: int, masks=None):
    """T steps; masks: None or a list/tensor [T, N, H, W]."""
    for t in range(T):
        m = None if masks is None else masks[t]
        p_un, p_burn = relaxed_step(p_un, p_burn, r, p_continue, m)
    return p_un, p_burn


def avg_pool(x: torch.Tensor, k: int) -> torch.Tensor:
    """Non-overlapping k x k average pooling of [N, H, W] (H, W multiples of k)."""
    N, H, W = x.shape
    return x.reshape(N, H // k, k, W // k, k).mean(dim=(2, 4))


def calibration_loss(p_un_T: torch.Tensor, target: torch.Tensor, pool: int = 4,
                     w_mse: float = 1.0) -> torch.Tensor:
    """Section 4: binary cross-entropy on the spread shape plus MSE after 2-D
    average pooling on the scale.  The prediction is the probability that a
    cell has caught fire, 1 - p_un.  The cross-entropy is PyTorch's (its logs
    are clamped at -100, so cells the fire never reaches are finite)."""
    pred = 1.0 - p_un_T
    bce = torch.nn.functional.binary_cross_entropy(pred, target)
    mse = ((avg_pool(pred, pool) - avg_pool(target, pool)) ** 2).mean()
    return bce + w_mse * mse


def straight_through_grad(states, r_of_theta, theta, a_un, a_burn):
    """Reference gradient of the straight-through rollout: the adjoint of the
    relaxed step (Eqs. 5-10) chained backward along a sampled discrete
    trajectory, each step linearised at the hard planes of the state before
    it (p_un = [no fuel or can burn], p_burn = [burning]).

    states: list of T int arrays [N, H, W] (the state before each step);
    r_of_theta(th) -> rates [N, H, W, 8] (FP64, differentiable in th);
    theta: FP64 parameter vector whose entry 5 is p_continue; a_un, a_burn:
    adjoints of the final planes.  Returns dL/dtheta."""
    a_u = torch.as_tensor(a_un, dtype=torch.float64)
    a_b = torch.as_tensor(a_burn, dtype=torch.float64)
    g = torch.zeros_like(theta, dtype=torch.float64)
    for x in reversed(states):
        x = torch.as_tensor(x)
        pu = (x <= 1).to(torch.float64).requires_grad_(True)
        pb = (x == 2).to(torch.float64).requires_grad_(True)
        th = theta.detach().clone().requires_grad_(True)
        ou, ob = relaxed_step(pu, pb, r_of_theta(th), th[5])
        L = (a_u * ou).sum() + (a_b * ob).sum()
        gu, gb, gt = torch.autograd.grad(L, [pu, pb, th])
        g = g + gt
        a_u, a_b = gu, gb
    return g
