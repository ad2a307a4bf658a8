"""jwf_step_relaxed_bwd_noalloc: the relaxed adjoint step for callers that
cannot allocate device memory (a framework's custom operator that hands over
its buffers and forbids allocation, a real-time loop that must not allocate
once running).

The entry point keeps its scratch in a file-scope device array, so two calls
in a row share (and reuse) that scratch.  Each call's outputs must match the
context entry point jwf_step_relaxed_bwd on the same inputs, within the
tolerance the adjoint parity tests use (1e-4 relative).  This file is named so
that pytest collects it last; it must pass both alone in a fresh process and
after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2512_06102_gb300 import jwf, scenarios
from tests.gpu_util import make_sim, require_gpu, to



def _close(g, ref, rel=1e-4, floor=1e-7):
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    tol = rel * np.abs(ref) + floor * np.abs(ref).max()
    assert (np.abs(g - ref) <= tol).all()


@pytest.mark.gpu
def test_noalloc_matches_context_entry_point_twice():
    require_gpu()
    N, H, W = 5, 96, 80
    scn = scenarios.make_scenario(H, W, N=N, seed=12)
    sim = make_sim(scn, keep_rates=True)
    sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    _, r = sim.probs()
    rng = np.random.default_rng(12)
    cells = N * H * W
    for call in range(2):
        pb = (rng.random(cells) < 0.1).astype(np.float32) * rng.random(cells).astype(np.float32)
        pu = ((1.0 - pb) * rng.random(cells)).astype(np.float32)
        au = rng.standard_normal(cells).astype(np.float32)
        ab = rng.standard_normal(cells).astype(np.float32)
        m = (rng.random(cells) < 0.05).astype(np.float32) * 0.7 if call == 1 else None
        args = [to(pu), to(pb), to(au), to(ab)]
        mask = None if m is None else to(m)
        gpc_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        gu_ref, gb_ref = sim.relaxed_bwd(*args, mask=mask, gpc=gpc_ref)
        gpc = torch.zeros(1, dtype=torch.float64, device="cuda")
        gu, gb = jwf.relaxed_bwd_noalloc(N, H, W, r, scn.params.p_continue, *args, mask=mask, gpc=gpc)
        torch.cuda.synchronize()
        _close(gu.cpu().numpy(), gu_ref.cpu().numpy())
        _close(gb.cpu().numpy(), gb_ref.cpu().numpy())
        assert gpc.item() == pytest.approx(gpc_ref.item(), rel=1e-5)
    sim.close()


@pytest.mark.gpu
def test_noalloc_rejects_oversized_batch():
    require_gpu()
    x = torch.zeros(8, device="cuda")
    r = torch.zeros(64, device="cuda")
    st = jwf.lib().jwf_step_relaxed_bwd_noalloc(
        jwf.NOALLOC_MAX_CELLS // 16 + 1, 4, 4, r.data_ptr(), ctypes.c_float(0.5), x.data_ptr(), x.data_ptr(),
        None, x.data_ptr(), x.data_ptr(), torch.zeros(8, device="cuda").data_ptr(),
        torch.zeros(8, device="cuda").data_ptr(), None, torch.cuda.current_stream().cuda_stream)
    assert st == 1                      # JWF_EINVAL, nothing launched


@pytest.mark.gpu
def test_noalloc_largest_batch_and_no_gpc():
    """The largest batch the scratch holds (one 2048 x 2048 grid, exactly
    JWF_NOALLOC_MAX_CELLS cells, so every thread of the capped grid loops
    eight times) without the p_continue output, twice in a row."""
    require_gpu()
    H = W = 2048
    assert H * W == jwf.NOALLOC_MAX_CELLS
    scn = scenarios.make_scenario(H, W, N=1, seed=13)
    sim = make_sim(scn, keep_rates=True)
    sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    _, r = sim.probs()
    g = torch.Generator(device="cuda").manual_seed(13)
    for call in range(2):
        pb = (torch.rand(H * W, device="cuda", generator=g) < 0.2).float() * torch.rand(H * W, device="cuda",
                                                                                          generator=g)
        pu = (1.0 - pb) * torch.rand(H * W, device="cuda", generator=g)
        au = torch.randn(H * W, device="cuda", generator=g)
        ab = torch.randn(H * W, device="cuda", generator=g)
        gu_ref, gb_ref = sim.relaxed_bwd(pu, pb, au, ab)
        gu, gb = jwf.relaxed_bwd_noalloc(1, H, W, r, scn.params.p_continue, pu, pb, au, ab)
        torch.cuda.synchronize()
        _close(gu.cpu().numpy(), gu_ref.cpu().numpy())
        _close(gb.cpu().numpy(), gb_ref.cpu().numpy())
    sim.close()


@pytest.mark.gpu
def test_noalloc_rejects_overlapping_buffers():
    """Outputs that share bytes with an input or with each other are refused
    on the host, before anything is launched."""
    require_gpu()
    cells = 4 * 8 * 8
    r = torch.zeros(8 * cells, device="cuda")
    x = torch.zeros(3 * cells, device="cuda")
    a, b = torch.zeros(cells, device="cuda"), torch.zeros(cells, device="cuda")
    gu, gb = torch.zeros(cells, device="cuda"), torch.zeros(cells, device="cuda")
    gpc = torch.zeros(1, dtype=torch.float64, device="cuda")
    P = lambda t: None if t is None else t.data_ptr()
    s = torch.cuda.current_stream().cuda_stream

    def call(pun, gun, gburn, gpc_):
        return jwf.lib().jwf_step_relaxed_bwd_noalloc(4, 8, 8, P(r), ctypes.c_float(0.5), P(pun), P(b), None,
                                                      P(a), P(b), P(gun), P(gburn), P(gpc_), s)

    assert call(x[:cells], x[cells // 2:cells // 2 + cells], gb, gpc) == 1     # d_gun half over d_pun
    assert call(a, gu, gu, gpc) == 1                                             # d_gun == d_gburn
    assert call(a, x[:cells], x[cells - 1:2 * cells - 1], gpc) == 1              # outputs share one float
    assert call(a, gu, gb, gu.view(torch.float64)[:1]) == 1                      # d_gpc inside d_gun
    assert call(a, gu, r[8 * cells - cells:], None) == 1                         # d_gburn inside d_r
    assert call(a, gu, gb, gpc) == 0                                             # disjoint: accepted
    torch.cuda.synchronize()


def test_noalloc_binding_checks_sizes_and_types():
    """The binding refuses buffers whose size or type does not match the call
    before any pointer reaches the library (runs without a GPU)."""
    n, H, W = 2, 4, 4
    c = n * H * W
    f = lambda k: torch.zeros(k, dtype=torch.float32)
    ok = dict(r=f(8 * c), pun=f(c), pburn=f(c), gun_out=f(c), gburn_out=f(c))
    bad = [dict(r=f(8 * c - 1)), dict(pun=f(c + 1)), dict(gburn_out=f(c - 1)),
           dict(pburn=torch.zeros(c, dtype=torch.float64)), dict(mask=f(c - 2)), dict(gun=f(2 * c)),
           dict(gpc=torch.zeros(1, dtype=torch.float32)), dict(gpc=torch.zeros(2, dtype=torch.float64))]
    for b in bad:
        kw = dict(ok, **b)
        r = kw.pop("r")
        with pytest.raises(ValueError):
            jwf.relaxed_bwd_noalloc(n, H, W, r, 0.5, kw.pop("pun"), kw.pop("pburn"), kw.pop("gun_out"),
                                    kw.pop("gburn_out"), **kw)
    with pytest.raises(ValueError):
        jwf.relaxed_bwd_noalloc(0, H, W, ok["r"], 0.5, ok["pun"], ok["pburn"], ok["gun_out"], ok["gburn_out"])
