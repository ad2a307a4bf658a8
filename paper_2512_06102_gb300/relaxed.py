"""Differentiable relaxed rollout (Section 3, Eqs. 5-10) on libjwf, and the
straight-through rollout (stochastic forward, relaxed backward).

`RelaxedRollout.apply(theta, p_un0, p_burn0, sim, scene, T, masks, ckpt_every)`
runs T relaxed steps with libjwf's forward kernel and returns (p_un_T,
p_burn_T); its backward runs libjwf's adjoint kernels step by step in reverse,
accumulates the rate adjoint over fixed step chunks (jwf_rates_accumulate)
and contracts it into parameter gradients once (jwf_rates_contract).  This
is the gradient the paper's calibration uses (Section 4: Adam on the
raw-probabilities routine).

theta (float64, any device) = [p_base, alpha_w1, alpha_w2, alpha_s,
alpha_gamma, p_continue, mu_veg[C], mu_den[C]].

Memory: `ckpt_every` = 0 keeps every state of the forward (2 x 4 B a cell
and step) and the backward recomputes nothing; k > 0 keeps the states at
every k-th step (k rounded up to a multiple of CHUNK) and the backward
recomputes one segment at a time; "sqrt" takes k = ceil(sqrt(T)); None (the
default) keeps every state when they take at most a quarter of the free
device memory, else uses "sqrt".  The rate adjoint is accumulated on
CHUNK-step blocks aligned to absolute step indices, so the gradients do not
depend on the choice (bit for bit).
"""
from __future__ import annotations

import math

import torch

from . import jwf

CHUNK = 16


def segment_length(T: int, ckpt_every) -> int:
    """Steps per checkpoint segment; T (one segment) when every state is kept."""
    if ckpt_every == 0:
        return max(T, 1)
    if ckpt_every is None or ckpt_every == "sqrt":
        ckpt_every = int(math.ceil(math.sqrt(max(T, 1))))
    s = max(CHUNK, int(math.ceil(int(ckpt_every) / CHUNK)) * CHUNK)
    return min(s, max(CHUNK, int(math.ceil(T / CHUNK)) * CHUNK))


def resolve_ckpt(T: int, cells: int, ckpt_every, device) -> int | str:
    """The checkpoint policy for a rollout of T steps on `cells` cells."""
    if ckpt_every is not None:
        return ckpt_every
    need = (T + 1) * cells * 2 * 4
    free, _ = torch.cuda.mem_get_info(device)
    return 0 if need <= free // 4 else "sqrt"


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
                ckpt_every=None, cell_size: float = 30.0):
        cls, dem, ws, wd = scene
        sim.set_params(theta_to_params(theta, sim.n_classes, cell_size))
        sim.precompute_probs(cls, dem, ws, wd)
        tables_version = sim.tables_version
        ckpt_every = resolve_ckpt(T, sim.cells, ckpt_every, p_un0.device)
        seg = segment_length(T, ckpt_every)
        pu, pb = p_un0.contiguous(), p_burn0.contiguous()
        if ckpt_every == 0:
            # keep every state: PU[t], PB[t] is the state before step t
            PU = torch.empty((T + 1, sim.cells), dtype=torch.float32, device=pu.device)
            PB = torch.empty_like(PU)
            PU[0].copy_(pu)
            PB[0].copy_(pb)
            if T > 0:
                sim.relaxed_fwd_steps(PU[0], PB[0], PU[1:], PB[1:], masks=None if masks is None else masks[:T])
            ctx.ckpts = [(PU, PB)]
            out_u, out_b = PU[T], PB[T]
        else:
            ckpts = []
            bu = torch.empty((seg, sim.cells), dtype=torch.float32, device=pu.device)
            bb = torch.empty_like(bu)
            cu, cb = pu.clone(), pb.clone()
            for a in range(0, T, seg):
                b = min(a + seg, T)
                ckpts.append((cu, cb))
                sim.relaxed_fwd_steps(cu, cb, bu[:b - a], bb[:b - a], masks=None if masks is None else masks[a:b])
                cu, cb = bu[b - a - 1].clone(), bb[b - a - 1].clone()
            ctx.ckpts = ckpts
            out_u, out_b = cu, cb
        ctx.sim, ctx.scene, ctx.T, ctx.masks, ctx.seg = sim, scene, T, masks, seg
        ctx.keep_all = ckpt_every == 0
        ctx.tables_version = tables_version
        ctx.theta_device = theta.device
        ctx.cell_size = cell_size
        ctx.theta = theta.detach().clone()
        return out_u.clone(), out_b.clone()

    @staticmethod
    def backward(ctx, g_un, g_burn):
        sim, T, seg, masks = ctx.sim, ctx.T, ctx.seg, ctx.masks
        cls, dem, ws, wd = ctx.scene
        # the context may have been used since the forward: restore its tables
        if sim.tables_version != ctx.tables_version:
            sim.set_params(theta_to_params(ctx.theta, sim.n_classes, ctx.cell_size))
            sim.precompute_probs(cls, dem, ws, wd)
        dev = g_un.device
        cells = sim.cells
        gparams = torch.zeros(sim.grad_size, dtype=torch.float64, device=dev)
        gpc = torch.zeros(1, dtype=torch.float64, device=dev)
        gu = (g_un if g_un is not None else torch.zeros(cells, device=dev)).contiguous().clone()
        gb = (g_burn if g_burn is not None else torch.zeros(cells, device=dev)).contiguous().clone()
        n_seg = (T + seg - 1) // seg if T > 0 else 0
        if not ctx.keep_all:
            pu_buf = torch.empty((seg, cells), dtype=torch.float32, device=dev)
            pb_buf = torch.empty((seg, cells), dtype=torch.float32, device=dev)
        glam = torch.empty((CHUNK, cells), dtype=torch.float32, device=dev)
        gr = torch.zeros((cells, 8), dtype=torch.float32, device=dev)     # rate adjoint
        ngu, ngb = torch.empty_like(gu), torch.empty_like(gb)
        for si in reversed(range(n_seg)):
            a = si * seg
            b = min(a + seg, T)
            if ctx.keep_all:
                PU, PB = ctx.ckpts[0]
                su, sb = PU[a:b], PB[a:b]
            else:
                # recompute the states p_a .. p_{b-1} from the checkpoint
                su, sb = pu_buf, pb_buf
                su[0].copy_(ctx.ckpts[si][0])
                sb[0].copy_(ctx.ckpts[si][1])
                if b - a > 1:
                    sim.relaxed_fwd_steps(su[0], sb[0], su[1:b - a], sb[1:b - a],
                                          masks=None if masks is None else masks[a:b - 1])
            # adjoint steps in reverse, one CHUNK-step block (aligned to
            # absolute step indices) a call; then its rate adjoint
            hi = b
            while hi > a:
                lo = max(a, ((hi - 1) // CHUNK) * CHUNK)
                mk = None if masks is None else masks[lo:hi]
                sim.relaxed_bwd_steps(su[lo - a:hi - a], sb[lo - a:hi - a], gu, gb, ngu, ngb, masks=mk,
                                      glam=glam[:hi - lo], gpc=gpc)
                gu, ngu = ngu, gu
                gb, ngb = ngb, gb
                sim.rates_accumulate(glam[:hi - lo], sb[lo - a:hi - a], gr, mask=mk)
                hi = lo
        sim.rates_contract(gr, cls, dem, ws, wd, gparams)
        C = sim.n_classes
        g = torch.empty(6 + 2 * C, dtype=torch.float64, device=dev)
        g[0:5] = gparams[0:5]
        g[5] = gpc[0]
        g[6:] = gparams[5:]
        return (g.to(ctx.theta_device), gu, gb, None, None, None, None, None, None)


def rollout(theta, p_un0, p_burn0, sim, scene, T, masks=None, ckpt_every=None, cell_size=30.0):
    return RelaxedRollout.apply(theta, p_un0, p_burn0, sim, scene, T, masks, ckpt_every, cell_size)


class StraightThroughRollout(torch.autograd.Function):
    """Straight-through rollout: the forward runs T steps of the stochastic
    update (Section 3) from the discrete states F0 and returns the hard planes
    (p_un_T, p_burn_T) of the sampled last state; the backward is the adjoint
    of the relaxed step (Eqs. 5-10) evaluated along the sampled trajectory
    (libjwf's adjoint kernels on jwf_state_planes of the recorded states),
    which gives gradients with respect to theta (the rates and p_continue).
    The sample depends on the context's seed (Sim.set_seed).

    With build_tables the context's tables are rebuilt from theta and the
    scene (the context needs JWF_KEEP_RATES); otherwise the caller's tables
    (jwf_set_probs with rates) are used as they are, and theta must match them
    for the gradient to mean anything."""

    @staticmethod
    def forward(ctx, theta, sim: jwf.Sim, scene, F0, T: int, build_tables: bool = True, cell_size: float = 30.0):
        cls, dem, ws, wd = scene
        if build_tables:
            sim.set_params(theta_to_params(theta, sim.n_classes, cell_size))
            sim.precompute_probs(cls, dem, ws, wd)
        hist = torch.empty((T, sim.cells), dtype=torch.uint8, device=F0.device)
        sim.load_state(F0)
        sim.step(T, None, history=hist)
        pu, pb = sim.state_planes(hist[T - 1:T])
        ctx.sim, ctx.scene, ctx.T, ctx.hist, ctx.F0 = sim, scene, T, hist, F0
        ctx.theta_device = theta.device
        return pu[0], pb[0]

    @staticmethod
    def backward(ctx, g_un, g_burn):
        sim, T = ctx.sim, ctx.T
        cls, dem, ws, wd = ctx.scene
        dev = ctx.F0.device
        cells = sim.cells
        states = torch.cat([ctx.F0.reshape(1, -1), ctx.hist[:T - 1]], 0)      # state before each step
        PU, PB = sim.state_planes(states)
        gparams = torch.zeros(sim.grad_size, dtype=torch.float64, device=dev)
        gpc = torch.zeros(1, dtype=torch.float64, device=dev)
        gu = (g_un if g_un is not None else torch.zeros(cells, device=dev)).contiguous().clone()
        gb = (g_burn if g_burn is not None else torch.zeros(cells, device=dev)).contiguous().clone()
        ngu, ngb = torch.empty_like(gu), torch.empty_like(gb)
        glam = torch.empty((CHUNK, cells), dtype=torch.float32, device=dev)
        gr = torch.zeros((cells, 8), dtype=torch.float32, device=dev)
        hi = T
        while hi > 0:
            lo = ((hi - 1) // CHUNK) * CHUNK
            sim.relaxed_bwd_steps(PU[lo:hi], PB[lo:hi], gu, gb, ngu, ngb, glam=glam[:hi - lo], gpc=gpc)
            gu, ngu = ngu, gu
            gb, ngb = ngb, gb
            sim.rates_accumulate(glam[:hi - lo], PB[lo:hi], gr)
            hi = lo
        sim.rates_contract(gr, cls, dem, ws, wd, gparams)
        C = sim.n_classes
        g = torch.empty(6 + 2 * C, dtype=torch.float64, device=dev)
        g[0:5] = gparams[0:5]
        g[5] = gpc[0]
        g[6:] = gparams[5:]
        return (g.to(ctx.theta_device), None, None, None, None, None, None)


def straight_through(theta, sim, scene, F0, T, build_tables=True, cell_size=30.0):
    return StraightThroughRollout.apply(theta, sim, scene, F0, T, build_tables, cell_size)


def calibration_loss(p_un_T: torch.Tensor, target: torch.Tensor, H: int, W: int, pool: int = 4,
                     w_mse: float = 1.0, n_total: int | None = None) -> torch.Tensor:
    """Section 4: binary cross-entropy on the spread shape plus MSE after 2-D
    average pooling; the prediction is 1 - p_un.  Uniform batches of H x W.

    Both terms are means over the whole batch.  A rank that holds n of the
    batch's n_total grids passes n_total: its value is then its share (the
    sums over its own grids divided by the whole batch's counts), and the
    shares of all ranks add up to the loss of the whole batch, as do their
    gradients.  n_total=None means this call sees the whole batch."""
    pred = (1.0 - p_un_T).reshape(-1, H, W)
    tgt = target.reshape(-1, H, W)
    n = pred.shape[0]
    n_all = n if n_total is None else int(n_total)
    if n_all < 1:
        raise ValueError("the batch holds no grids")
    bce = torch.nn.functional.binary_cross_entropy(pred, tgt, reduction="sum") / float(n_all * H * W)
    pp = pred.reshape(n, H // pool, pool, W // pool, pool).mean(dim=(2, 4))
    tp = tgt.reshape(n, H // pool, pool, W // pool, pool).mean(dim=(2, 4))
    mse = ((pp - tp) ** 2).sum() / float(n_all * (H // pool) * (W // pool))
    return bce + w_mse * mse
