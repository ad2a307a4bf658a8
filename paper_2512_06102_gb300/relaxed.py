"""Differentiable relaxed rollout (Section 3, Eqs. 5-10) on libjwf.

`RelaxedRollout.apply(theta, p_un0, p_burn0, sim, scene, T, masks, ckpt_every)`
runs T relaxed steps with libjwf's forward kernel and returns (p_un_T,
p_burn_T); its backward runs libjwf's adjoint kernels step by step in reverse,
accumulates the rate adjoint over fixed step chunks (jwf_rates_accumulate)
and contracts it into parameter gradients once (jwf_rates_contract).  This
is the gradient the paper's calibration uses (Section 4: Adam on the
raw-probabilities routine).

theta (float64, any device) = [p_base, alpha_w1, alpha_w2, alpha_s,
alpha_gamma, p_continue, mu_veg[C], mu_den[C]].

Memory: only the states at every `ckpt_every`-th step are kept by the
forward; the backward recomputes one segment at a time (default segment
ceil(sqrt(T)) rounded up to a multiple of CHUNK).  The rate adjoint is
accumulated on CHUNK-step blocks aligned to absolute step indices, so
checkpointed and non-checkpointed gradients are bit-identical.
"""
from __future__ import annotations

import math

import torch

from . import jwf

CHUNK = 8


def segment_length(T: int, ckpt_every: int | None) -> int:
    if ckpt_every is None:
        ckpt_every = int(math.ceil(math.sqrt(max(T, 1))))
    s = max(CHUNK, int(math.ceil(ckpt_every / CHUNK)) * CHUNK)
    return min(s, max(CHUNK, int(math.ceil(T / CHUNK)) * CHUNK))


def theta_to_params(theta: torch.Tensor, n_classes: int, cell_size: float = 30.0) -> jwf.ParamSet:
    v = theta.detach().double().cpu().tolist()
    C = n_classes
    import numpy as np
    return jwf.ParamSet(p_base=v[0], alpha_w1=v[1], alpha_w2=v[2], alpha_s=v[3], alpha_gamma=v[4],
                        p_continue=v[5], cell_size=cell_size,
                        mu_veg=np.array(v[6:6 + C], np.float32), mu_den=np.array(v[6 + C:6 + 2 * C], np.float32))


class RelaxedRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, p_un0, p_burn0, sim: jwf.Sim, scene, T: int, masks=None,
                ckpt_every: int | None = None, cell_size: float = 30.0):
        cls, dem, ws, wd = scene
        sim.set_params(theta_to_params(theta, sim.n_classes, cell_size))
        sim.precompute_probs(cls, dem, ws, wd)
        seg = segment_length(T, ckpt_every)
        pu, pb = p_un0.contiguous(), p_burn0.contiguous()
        ckpts = []
        bu, bb = torch.empty_like(pu), torch.empty_like(pb)
        for t in range(T):
            if t % seg == 0:
                ckpts.append((pu.clone(), pb.clone()))
            m = None if masks is None else masks[t]
            sim.relaxed_fwd(pu, pb, m, bu, bb)
            if t == 0:
                pu, pb = bu, bb
                bu, bb = torch.empty_like(pu), torch.empty_like(pb)
            else:
                pu, bu = bu, pu
                pb, bb = bb, pb
        ctx.sim, ctx.scene, ctx.T, ctx.masks, ctx.seg = sim, scene, T, masks, seg
        ctx.ckpts = ckpts
        ctx.theta_device = theta.device
        ctx.cell_size = cell_size
        ctx.theta = theta.detach().clone()
        return pu.clone(), pb.clone()

    @staticmethod
    def backward(ctx, g_un, g_burn):
        sim, T, seg, masks = ctx.sim, ctx.T, ctx.seg, ctx.masks
        cls, dem, ws, wd = ctx.scene
        # the context may have been used since the forward: restore its tables
        sim.set_params(theta_to_params(ctx.theta, sim.n_classes, ctx.cell_size))
        sim.precompute_probs(cls, dem, ws, wd)
        dev = g_un.device
        cells = sim.cells
        gparams = torch.zeros(sim.grad_size, dtype=torch.float64, device=dev)
        gpc = torch.zeros(1, dtype=torch.float64, device=dev)
        gu = (g_un if g_un is not None else torch.zeros(cells, device=dev)).contiguous().clone()
        gb = (g_burn if g_burn is not None else torch.zeros(cells, device=dev)).contiguous().clone()
        n_seg = len(ctx.ckpts)
        pu_buf = torch.empty((seg, cells), dtype=torch.float32, device=dev)
        pb_buf = torch.empty((seg, cells), dtype=torch.float32, device=dev)
        glam = torch.empty((seg, cells), dtype=torch.float32, device=dev)
        gr = torch.zeros((cells, 8), dtype=torch.float32, device=dev)     # rate adjoint
        mk_buf = None if masks is None else torch.empty((seg, cells), dtype=torch.float32, device=dev)
        ngu, ngb = torch.empty_like(gu), torch.empty_like(gb)
        for si in reversed(range(n_seg)):
            a = si * seg
            b = min(a + seg, T)
            # recompute the states p_a .. p_{b-1} from the checkpoint
            pu_buf[0].copy_(ctx.ckpts[si][0])
            pb_buf[0].copy_(ctx.ckpts[si][1])
            for t in range(a, b - 1):
                m = None if masks is None else masks[t]
                sim.relaxed_fwd(pu_buf[t - a], pb_buf[t - a], m, pu_buf[t - a + 1], pb_buf[t - a + 1])
            if masks is not None:
                mk_buf[:b - a].copy_(masks[a:b])
            # adjoint steps in reverse; rate contraction per aligned CHUNK
            hi = b
            for t in reversed(range(a, b)):
                m = None if masks is None else masks[t]
                sim.relaxed_bwd(pu_buf[t - a], pb_buf[t - a], gu, gb, m, ngu, ngb, glam[t - a], gpc)
                gu, ngu = ngu, gu
                gb, ngb = ngb, gb
                if t % CHUNK == 0:
                    lo = t
                    sim.rates_accumulate(glam[lo - a:hi - a], pb_buf[lo - a:hi - a], gr,
                                         mask=None if masks is None else mk_buf[lo - a:hi - a])
                    hi = lo
            assert hi == a
        sim.rates_contract(gr, cls, dem, ws, wd, gparams)
        C = sim.n_classes
        g = torch.empty(6 + 2 * C, dtype=torch.float64, device=dev)
        g[0:5] = gparams[0:5]
        g[5] = gpc[0]
        g[6:] = gparams[5:]
        return (g.to(ctx.theta_device), gu, gb, None, None, None, None, None, None)


def rollout(theta, p_un0, p_burn0, sim, scene, T, masks=None, ckpt_every=None, cell_size=30.0):
    return RelaxedRollout.apply(theta, p_un0, p_burn0, sim, scene, T, masks, ckpt_every, cell_size)


def calibration_loss(p_un_T: torch.Tensor, target: torch.Tensor, H: int, W: int, pool: int = 4,
                     w_mse: float = 1.0) -> torch.Tensor:
    """Section 4: binary cross-entropy on the spread shape plus MSE after 2-D
    average pooling; the prediction is 1 - p_un.  Uniform batches of H x W."""
    pred = (1.0 - p_un_T).reshape(-1, H, W)
    tgt = target.reshape(-1, H, W)
    bce = torch.nn.functional.binary_cross_entropy(pred, tgt)
    n = pred.shape[0]
    pp = pred.reshape(n, H // pool, pool, W // pool, pool).mean(dim=(2, 4))
    tp = tgt.reshape(n, H // pool, pool, W // pool, pool).mean(dim=(2, 4))
    return bce + w_mse * ((pp - tp) ** 2).mean()
