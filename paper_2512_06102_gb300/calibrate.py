"""Gradient-based calibration of the spread parameters (Section 4).

Targets are burn maps: the fraction of seeded runs of the stochastic step
(Section 3) in which a cell has caught fire (burning or burned) after T
steps.  The fit runs the relaxed rollout (Eqs. 5-10) from the same initial
fires, takes the Section 4 loss (BCE on the spread shape + MSE after average
pooling) and updates the free parameters with Adam, as the paper does with
its raw-probabilities routine.  Under torch.distributed each rank holds a
shard of the grids and evaluates its share of the whole batch's loss; the
shares' gradients (and values) are summed over ranks before the update, so
every rank takes the same step as a single process holding the whole batch.

theta layout (float64): [p_base, alpha_w1, alpha_w2, alpha_s, alpha_gamma,
p_continue, mu_veg[C], mu_den[C]].  By default p_base, the two wind
coefficients, the slope coefficient and mu_veg are free; alpha_gamma (it
enters only as a product with p_base), p_continue and mu_den (no-fuel classes
sit at -1) stay fixed.
"""
from __future__ import annotations

import numpy as np
import torch

from . import jwf, relaxed, shard


def theta_of(params, n_classes: int) -> torch.Tensor:
    p = jwf.ParamSet.from_any(params)
    return torch.tensor([p.p_base, p.alpha_w1, p.alpha_w2, p.alpha_s, p.alpha_gamma, p.p_continue]
                        + [float(x) for x in p.mu_veg[:n_classes]] + [float(x) for x in p.mu_den[:n_classes]],
                        dtype=torch.float64)


def default_free(n_classes: int) -> torch.Tensor:
    """Mask of the parameters the fit moves (see the module docstring)."""
    m = torch.zeros(6 + 2 * n_classes, dtype=torch.float64)
    m[0:4] = 1.0
    m[6:6 + n_classes] = 1.0
    return m


def burn_maps(H: int, W: int, n_envs: int, params, scene, F0: torch.Tensor, T: int, seeds=(0, 1, 2, 3, 4),
              drops: torch.Tensor | None = None) -> torch.Tensor:
    """Mean over seeds of [state is burning or burned] after T stochastic
    steps (float32 [cells], on F0's device)."""
    acc = torch.zeros(F0.shape[0], dtype=torch.float32, device=F0.device)
    for s in seeds:
        sim = jwf.Sim(H, W, n_envs=n_envs, n_classes=len(jwf.ParamSet.from_any(params).mu_veg), seed=int(s))
        try:
            sim.set_params(params)
            sim.set_terrain(*scene)
            sim.set_kernel(jwf.KERNEL_FUSED)
            sim.load_state(F0)
            sim.step(T, drops)
            acc += (sim.state() >= 2).to(torch.float32)
        finally:
            sim.close()
    return acc / float(len(seeds))


def sharded_loss_grad(z: torch.Tensor, local_loss: torch.Tensor | None, free: torch.Tensor) -> float:
    """Backward of this rank's share of the whole-batch loss (None when the
    rank holds no grids), restricted to the free parameters and summed over
    ranks into z.grad; returns the whole batch's loss."""
    if local_loss is not None:
        local_loss.backward()
        lv = local_loss.detach().to(torch.float64)
    else:
        lv = torch.zeros((), dtype=torch.float64)
    if z.grad is None:
        z.grad = torch.zeros_like(z)
    g = z.grad.detach()
    g.mul_(free.to(g.device))
    return shard.reduce_loss_and_grad_(g, lv.to(g.device))


def fit(sim: jwf.Sim | None, scene, F0: torch.Tensor, target: torch.Tensor, theta0: torch.Tensor, T: int,
        iters: int = 100, lr: float = 0.05, free: torch.Tensor | None = None, pool: int = 4,
        ckpt_every=None, callback=None):
    """Adam on the free parameters of theta, in steps relative to each
    parameter's size; returns (theta, [whole-batch loss per iteration]).  sim
    must have been created with keep_rates=True and hold a uniform batch (the
    pooled loss reshapes to [N, H, W]).  Under torch.distributed every rank
    calls fit with its own shard; a rank whose shard is empty passes
    sim=None (scene, F0 and target are then ignored) and still takes part in
    every reduction."""
    theta0 = theta0.detach().to(torch.float64)
    n_classes = (theta0.numel() - 6) // 2
    if sim is not None:
        H, W = int(sim.H[0]), int(sim.W[0])
        if not (np.all(sim.H == H) and np.all(sim.W == W)):
            raise ValueError("calibration needs a uniform batch")
        pb0 = (F0 == 2).to(torch.float32)
        pu0 = 1.0 - pb0
        cell_size = sim.params.cell_size if sim.params is not None else 30.0
    n_total = shard.global_count(0 if sim is None else sim.N)
    free = default_free(n_classes) if free is None else free
    # Adam steps in units of each parameter's own size (the coefficients span
    # two orders of magnitude): theta = theta0 + scale * z
    scale = theta0.abs().clamp_min(0.05)
    z = torch.zeros_like(theta0, requires_grad=True)
    opt = torch.optim.Adam([z], lr=lr)
    losses = []
    for it in range(iters):
        opt.zero_grad()
        theta = theta0 + scale * z
        loss = None
        if sim is not None:
            ou, _ = relaxed.rollout(theta, pu0, pb0, sim, scene, T, ckpt_every=ckpt_every, cell_size=cell_size)
            loss = relaxed.calibration_loss(ou, target, H, W, pool=pool, n_total=n_total)
        losses.append(sharded_loss_grad(z, loss, free))
        opt.step()
        if callback is not None:
            callback(it, (theta0 + scale * z).detach(), losses[-1])
    return (theta0 + scale * z).detach(), losses
