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

pytestmark = pytest.mark.gpu


def _close(g, ref, rel=1e-4, floor=1e-7):
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    tol = rel * np.abs(ref) + floor * np.abs(ref).max()
    assert (np.abs(g - ref) <= tol).all()


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


def test_noalloc_rejects_oversized_batch():
    require_gpu()
    x = torch.zeros(8, device="cuda")
    r = torch.zeros(64, device="cuda")
    st = jwf.lib().jwf_step_relaxed_bwd_noalloc(
        jwf.NOALLOC_MAX_CELLS // 16 + 1, 4, 4, r.data_ptr(), ctypes.c_float(0.5), x.data_ptr(), x.data_ptr(),
        None, x.data_ptr(), x.data_ptr(), torch.zeros(8, device="cuda").data_ptr(),
        torch.zeros(8, device="cuda").data_ptr(), None, torch.cuda.current_stream().cuda_stream)
    assert st == 1                      # JWF_EINVAL, nothing launched
