"""Relaxed (raw-probabilities) step on the GPU against the FP64 oracle.

  * forward: one step within 1e-6 absolute; T = 100 steps within 1e-5 absolute
    (FP32 state against FP64);
  * one adjoint step: every input adjoint and dL/dp_continue within 1e-4
    relative of the oracle's autograd;
  * rollout gradients with respect to every parameter (T = 40) and to the
    initial maps (T = 12) within 1e-4 relative of the oracle's autograd (which
    the CPU suite pins to central differences), with tanker masks, on several
    tiles and a ragged tail;
  * the rate-adjoint accumulation (sum over steps of lambda-bar times the
    masked source burn probability) within 1e-6 relative, and its contraction
    with dr/dtheta within 1e-4 relative of the oracle's autograd; the one-call
    jwf_rates_bwd agrees with the two halves;
  * checkpointed and non-checkpointed gradients are bit-identical, and the
    multi-step calls equal the single-step calls bit for bit;
  * the tiled kernels (fused adjoint) and the plain one-thread-per-cell
    kernels (two-pass adjoint) agree to float rounding on a ragged batch;
  * T = 1000 on the 256 x 128^2 differentiation workload with sqrt(T)
    checkpoints: the parameter gradient of a loss on a sample of envs equals
    the oracle's for those envs, and every map entry is finite (the adjoint
    saturates at 1e35 instead of overflowing).
Parameter components are compared as |g - g_ref| <= 1e-4 |g_ref| + 1e-7 max|g_ref|
(the floor covers components that cancel to near zero).  Map entries are
compared as |g - g_ref| <= 1e-4 |g_ref| + 10 |g_ref32 - g_ref|, where g_ref32
is the same oracle evaluated in float32: a few entries cancel to values far
below their terms, and float32 arithmetic cannot resolve them any better
(the float32 oracle misses them too).  The map gradient is tested at a short
horizon on purpose: a spark ahead of the front grows about sum_d r per step,
so d p_T / d p_burn_0 leaves the float range after ~20 steps and, by T ~ 100,
its conditioning exceeds 1/eps_float with respect to the forward states
themselves (an FP64 adjoint over float states misses the FP64 reference by
orders of magnitude there), while the parameter gradient stays well
conditioned.
"""
import numpy as np
import pytest
import torch

from oracle import prob
from oracle import relaxed as orelaxed
from paper_2512_06102_gb300 import relaxed, scenarios
from tests.gpu_util import make_sim, oracle_tables, require_gpu, to

pytestmark = pytest.mark.gpu
f64 = torch.float64


def _planes(scn, rng, soft=True):
    F0 = scn.F0
    fuel = (F0 != 0).astype(np.float64)
    if soft:
        pb = np.where(F0 == 2, 1.0, 0.0) + fuel * (rng.random(F0.size) < 0.02) * rng.random(F0.size) * 0.5
        pb = np.minimum(pb, 1.0) * fuel
        pu = fuel * (1 - pb) * (0.7 + 0.3 * rng.random(F0.size)) + (1 - fuel)
    else:
        pb = (F0 == 2).astype(np.float64)
        pu = 1.0 - pb
    return pu, pb


def _oracle_rates(scn):
    return torch.as_tensor(oracle_tables(scn)[3]).reshape(scn.N, int(scn.H[0]), int(scn.W[0]), 8)


def test_forward_one_step_and_T100():
    require_gpu()
    scn = scenarios.make_scenario(128, 128, N=6, seed=1)
    rng = np.random.default_rng(0)
    pu, pb = _planes(scn, rng)
    sim = make_sim(scn, keep_rates=True)
    sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    r64 = _oracle_rates(scn)
    shp = (scn.N, 128, 128)
    m = (rng.random(scn.F0.size) < 0.01).astype(np.float32) * 0.8
    gu, gb = sim.relaxed_fwd(to(pu.astype(np.float32)), to(pb.astype(np.float32)), to(m))
    ou, ob = orelaxed.relaxed_step(torch.as_tensor(pu.astype(np.float32).astype(np.float64)).reshape(shp),
                                   torch.as_tensor(pb.astype(np.float32).astype(np.float64)).reshape(shp),
                                   r64, float(np.float32(scn.params.p_continue)),
                                   torch.as_tensor(m.astype(np.float64)).reshape(shp))
    assert np.abs(gu.cpu().numpy() - ou.reshape(-1).numpy()).max() < 1e-6
    assert np.abs(gb.cpu().numpy() - ob.reshape(-1).numpy()).max() < 1e-6
    # 100 steps
    pu_g, pb_g = to(pu.astype(np.float32)), to(pb.astype(np.float32))
    for _ in range(100):
        pu_g, pb_g = sim.relaxed_fwd(pu_g, pb_g)
    ou, ob = orelaxed.relaxed_rollout(torch.as_tensor(pu.astype(np.float32).astype(np.float64)).reshape(shp),
                                      torch.as_tensor(pb.astype(np.float32).astype(np.float64)).reshape(shp),
                                      r64, float(np.float32(scn.params.p_continue)), 100)
    err_u = np.abs(pu_g.cpu().numpy() - ou.reshape(-1).numpy()).max()
    err_b = np.abs(pb_g.cpu().numpy() - ob.reshape(-1).numpy()).max()
    assert err_u < 1e-5 and err_b < 1e-5, (err_u, err_b)
    pbd = 1 - pu_g - pb_g
    assert pbd.min().item() > -1e-5


def _close(g, ref, rel=1e-4, floor=1e-7, atol=0.0):
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    tol = rel * np.abs(ref) + floor * np.abs(ref).max() + atol
    bad = np.abs(g - ref) > tol
    assert not bad.any(), f"{bad.sum()} off; worst {np.max(np.abs(g - ref) / np.maximum(np.abs(ref), 1e-300))}"


def test_one_adjoint_step():
    require_gpu()
    scn = scenarios.make_scenario(96, 80, N=3, seed=2)
    rng = np.random.default_rng(1)
    pu, pb = _planes(scn, rng)
    pu32, pb32 = pu.astype(np.float32), pb.astype(np.float32)
    au = rng.standard_normal(pu.size).astype(np.float32)
    ab = rng.standard_normal(pu.size).astype(np.float32)
    m = (rng.random(pu.size) < 0.05).astype(np.float32) * rng.random(pu.size).astype(np.float32)
    sim = make_sim(scn, keep_rates=True)
    sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    gpc = torch.zeros(1, dtype=f64, device="cuda")
    glam = torch.empty(pu.size, device="cuda")
    gu, gb = sim.relaxed_bwd(to(pu32), to(pb32), to(au), to(ab), mask=to(m), glam=glam, gpc=gpc)
    # oracle: autograd of one FP64 step
    shp = (scn.N, 96, 80)
    U = torch.as_tensor(pu32.astype(np.float64)).reshape(shp).requires_grad_(True)
    B = torch.as_tensor(pb32.astype(np.float64)).reshape(shp).requires_grad_(True)
    pc = torch.tensor(float(np.float32(scn.params.p_continue)), dtype=f64, requires_grad=True)
    r64 = _oracle_rates(scn).requires_grad_(True)
    ou, ob = orelaxed.relaxed_step(U, B, r64, pc, torch.as_tensor(m.astype(np.float64)).reshape(shp))
    L = (torch.as_tensor(au.astype(np.float64)).reshape(shp) * ou).sum() + \
        (torch.as_tensor(ab.astype(np.float64)).reshape(shp) * ob).sum()
    rU, rB, rpc = torch.autograd.grad(L, [U, B, pc])
    torch.cuda.synchronize()
    _close(gu.cpu().numpy(), rU.reshape(-1).numpy())
    _close(gb.cpu().numpy(), rB.reshape(-1).numpy())
    assert gpc.item() == pytest.approx(rpc.item(), rel=1e-5)


def _theta(params, C):
    return torch.tensor([params.p_base, params.alpha_w1, params.alpha_w2, params.alpha_s, params.alpha_gamma,
                         params.p_continue] + list(params.mu_veg[:C]) + list(params.mu_den[:C]), dtype=f64)


def _oracle_grad(scn, theta, pu, pb, T, wu, wb, masks=None, envs=None, dtype=f64):
    """Gradient of sum(wu * p_un_T + wb * p_burn_T) by the oracle (FP64 by
    default; float32 only to gauge each entry's float32 conditioning).  The
    rates are always built in FP64."""
    C = len(scn.params.mu_veg)
    idx = range(scn.N) if envs is None else envs
    th = theta.clone().requires_grad_(True)
    U = torch.as_tensor(np.stack([scn.env(e, pu) for e in idx])).to(dtype).requires_grad_(True)
    B = torch.as_tensor(np.stack([scn.env(e, pb) for e in idx])).to(dtype).requires_grad_(True)
    cls = torch.as_tensor(np.stack([scn.env(e, scn.cls) for e in idx])).long()
    dem = torch.as_tensor(np.stack([scn.env(e, scn.dem) for e in idx]).astype(np.float64))
    sel = list(idx)
    r = prob.rates(cls, dem, torch.as_tensor(scn.wind_speed[sel].astype(np.float64)),
                   torch.as_tensor(scn.wind_dir[sel].astype(np.float64)), th[0], th[1], th[2], th[3], th[4],
                   th[6:6 + C], th[6 + C:6 + 2 * C], scn.params.cell_size).to(dtype)
    mk = None if masks is None else [torch.as_tensor(np.stack([scn.env(e, masks[t]) for e in idx])).to(dtype)
                                     for t in range(T)]
    ou, ob = orelaxed.relaxed_rollout(U, B, r, th[5].to(dtype), T, mk)
    WU = torch.as_tensor(np.stack([scn.env(e, wu) for e in idx])).to(dtype)
    WB = torch.as_tensor(np.stack([scn.env(e, wb) for e in idx])).to(dtype)
    L = (WU * ou).sum() + (WB * ob).sum()
    return [g.double() for g in torch.autograd.grad(L, [th, U, B])]


@pytest.mark.parametrize("T,check_maps", [(40, False), (12, True)])
def test_rollout_gradient_matches_oracle(T, check_maps):
    require_gpu()
    H, W, N = 70, 66, 3                 # several 256-cell tiles and a ragged tail
    scn = scenarios.make_scenario(H, W, N=N, seed=3)
    rng = np.random.default_rng(3)
    pu, pb = _planes(scn, rng)
    pu = pu.astype(np.float32).astype(np.float64)
    pb = pb.astype(np.float32).astype(np.float64)
    wu = rng.standard_normal(pu.size).astype(np.float32)
    wb = rng.standard_normal(pu.size).astype(np.float32)
    masks = (rng.random((T, pu.size)) < 0.01).astype(np.float32) * 0.9
    C = scenarios.N_CLASSES
    theta = _theta(scn.params, C)
    theta32 = theta.float().double()       # the GPU sees float32 parameters
    sim = make_sim(scn, keep_rates=True)
    scene = (to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    th = theta32.clone().requires_grad_(True)
    U = to(pu.astype(np.float32)).requires_grad_(True)
    B = to(pb.astype(np.float32)).requires_grad_(True)
    ou, ob = relaxed.rollout(th, U, B, sim, scene, T, masks=to(masks), ckpt_every=16)
    L = (to(wu) * ou).sum() + (to(wb) * ob).sum()
    gth, gU, gB = torch.autograd.grad(L, [th, U, B])
    rth, rU, rB = _oracle_grad(scn, theta32, pu, pb, T, wu, wb, masks=masks)
    _close(gth.cpu().numpy(), rth.numpy())
    if check_maps:
        _, sU, sB = _oracle_grad(scn, theta32, pu, pb, T, wu, wb, masks=masks, dtype=torch.float32)
        for g, ref, ref32 in ((gU, rU, sU), (gB, rB, sB)):
            ref = ref.reshape(-1).numpy()
            noise = np.abs(ref32.reshape(-1).numpy() - ref)
            _close(g.cpu().numpy(), ref, floor=0.0, atol=10.0 * noise + 1e-20)


def test_rate_adjoint_accumulate_and_contract():
    require_gpu()
    H, W, N, T = 70, 66, 3, 5
    scn = scenarios.make_scenario(H, W, N=N, seed=6)
    rng = np.random.default_rng(6)
    cells = N * H * W
    glam = rng.standard_normal((T, cells)).astype(np.float32)
    pb = rng.random((T, cells)).astype(np.float32)
    m = ((rng.random((T, cells)) < 0.1) * rng.random((T, cells))).astype(np.float32)
    sim = make_sim(scn, keep_rates=True)
    scene = (to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    sim.precompute_probs(*scene)
    gr = torch.zeros((cells, 8), dtype=torch.float32, device="cuda")
    sim.rates_accumulate(to(glam[:2]), to(pb[:2]), gr, mask=to(m[:2]))
    sim.rates_accumulate(to(glam[2:]), to(pb[2:]), gr, mask=to(m[2:]))
    gp = torch.zeros(sim.grad_size, dtype=f64, device="cuda")
    sim.rates_contract(gr, *scene, gp)
    gp1 = torch.zeros(sim.grad_size, dtype=f64, device="cuda")
    sim.rates_bwd(to(glam), to(pb), *scene, gp1, mask=to(m))
    # oracle: gr[v, d] = sum_t glam_t(v) (1 - m_t(u)) pb_t(u), u = v - Delta_d
    shp = (T, N, H, W)
    G = torch.as_tensor(glam.astype(np.float64)).reshape(shp)
    PB = torch.as_tensor(((1.0 - m.astype(np.float64)) * pb.astype(np.float64))).reshape(shp)
    ref = torch.stack([(G * prob.shift_from_source(PB, d)).sum(0) for d in range(8)], -1)
    got = gr.cpu().double().reshape(N, H, W, 8)
    scale = (G.abs() * prob.shift_from_source(PB.abs(), 0)).sum(0).max()
    assert torch.allclose(got, ref, rtol=1e-6, atol=1e-6 * float(scale))
    # contraction: d/dtheta sum_{v,d} gr[v, d] r(v, d; theta) with the GPU's gr
    C = scenarios.N_CLASSES
    th = _theta(scn.params, C).float().double().requires_grad_(True)
    r = prob.rates(torch.as_tensor(scn.cls).long().reshape(N, H, W),
                   torch.as_tensor(scn.dem.astype(np.float64)).reshape(N, H, W),
                   torch.as_tensor(scn.wind_speed.astype(np.float64)),
                   torch.as_tensor(scn.wind_dir.astype(np.float64)), th[0], th[1], th[2], th[3], th[4],
                   th[6:6 + C], th[6 + C:6 + 2 * C], scn.params.cell_size)
    (gth,) = torch.autograd.grad((got * r).sum(), [th])
    rg = torch.cat([gth[0:5], gth[6:]]).numpy()
    torch.cuda.synchronize()
    _close(gp.cpu().numpy(), rg)
    _close(gp1.cpu().numpy(), rg)


def test_checkpointing_is_bit_identical():
    require_gpu()
    scn = scenarios.make_scenario(64, 64, N=4, seed=4)
    rng = np.random.default_rng(4)
    pu, pb = _planes(scn, rng)
    T = 67
    wu = to(rng.standard_normal(pu.size).astype(np.float32))
    sim = make_sim(scn, keep_rates=True)
    scene = (to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    grads = []
    for ck in (0, 8, 16, 24, T, "sqrt"):
        th = _theta(scn.params, scenarios.N_CLASSES).float().double().requires_grad_(True)
        U = to(pu.astype(np.float32)).requires_grad_(True)
        B = to(pb.astype(np.float32)).requires_grad_(True)
        ou, ob = relaxed.rollout(th, U, B, sim, scene, T, ckpt_every=ck)
        L = (wu * ou).sum() + ob.sum()
        grads.append(torch.autograd.grad(L, [th, U, B]))
    for g in grads[1:]:
        for a, b in zip(grads[0], g):
            assert torch.equal(a, b)


def test_tiled_and_plain_kernels_agree():
    require_gpu()
    from paper_2512_06102_gb300 import jwf
    H = np.array([70, 33, 128, 17], np.int32)
    W = np.array([66, 150, 64, 5], np.int32)
    scn = scenarios.make_scenario(H, W, N=4, seed=8)
    rng = np.random.default_rng(8)
    pu, pb = _planes(scn, rng)
    n = pu.size
    au = to(rng.standard_normal(n).astype(np.float32))
    ab = to(rng.standard_normal(n).astype(np.float32))
    m = to((rng.random(n) < 0.05).astype(np.float32) * 0.7)
    sim = make_sim(scn, keep_rates=True)
    sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    out = {}
    for kern in (jwf.RELAXED_TILED, jwf.RELAXED_PLAIN):
        sim.set_relaxed_kernel(kern)
        ou, ob = sim.relaxed_fwd(to(pu.astype(np.float32)), to(pb.astype(np.float32)), m)
        gpc = torch.zeros(1, dtype=f64, device="cuda")
        glam = torch.empty(n, device="cuda")
        gu, gb = sim.relaxed_bwd(to(pu.astype(np.float32)), to(pb.astype(np.float32)), au, ab, mask=m,
                                 glam=glam, gpc=gpc)
        out[kern] = [x.cpu().double() for x in (ou, ob, gu, gb, glam)] + [gpc.cpu()]
    sim.set_relaxed_kernel(jwf.RELAXED_TILED)
    for a, b in zip(out[jwf.RELAXED_TILED][:5], out[jwf.RELAXED_PLAIN][:5]):
        assert torch.allclose(a, b, rtol=1e-6, atol=1e-7 * float(b.abs().max()))
    # dL/dp_continue: the sweep sums a_b pb in float over a strip's 32 cells a lane before the FP64 total,
    # the plain kernel in FP64 per cell; both within FP32 rounding of the sum of |a_b pb|
    scale = float((ab.abs().double() * (to(pb.astype(np.float32)) * (1 - m)).double()).sum())
    assert abs(out[jwf.RELAXED_TILED][5].item() - out[jwf.RELAXED_PLAIN][5].item()) <= 1e-6 * scale


@pytest.mark.parametrize("shape,T,with_masks", [((40, 72), 5, True), ((40, 72), 4, False),
                                                 (([17, 50, 33], [45, 100, 32]), 7, True),
                                                 (([16, 70], [31, 64]), 6, False),
                                                 (([1, 3, 130], [29, 2, 57]), 2, True),
                                                 ((128, 128), 16, False)])
def test_multi_step_calls_equal_single_steps(shape, T, with_masks):
    """jwf_relaxed_fwd_steps and jwf_relaxed_bwd_steps (two steps a pass on
    the tiled path, one for an odd step count's last step) equal single steps
    bit for bit, on ragged grids whose edges cut the 16 x 32 forward tiles and
    the 28- and 30-column adjoint strips; dL/dp_continue, summed per strip in
    another grouping, to float rounding."""
    require_gpu()
    if np.isscalar(shape[0]):
        scn = scenarios.make_scenario(shape[0], shape[1], N=3, seed=9)
    else:
        scn = scenarios.make_scenario(shape[0], shape[1], seed=9)
    rng = np.random.default_rng(9)
    pu, pb = _planes(scn, rng)
    n = pu.size
    masks = to(((rng.random((T, n)) < 0.05) * 0.8).astype(np.float32)) if with_masks else None
    sim = make_sim(scn, keep_rates=True)
    sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    U0, B0 = to(pu.astype(np.float32)), to(pb.astype(np.float32))
    SU = torch.empty((T, n), device="cuda")
    SB = torch.empty((T, n), device="cuda")
    sim.relaxed_fwd_steps(U0, B0, SU, SB, masks=masks)
    u, b = U0, B0
    states = [(U0, B0)]
    for t in range(T):
        u, b = sim.relaxed_fwd(u, b, None if masks is None else masks[t])
        assert torch.equal(u, SU[t]) and torch.equal(b, SB[t])
        states.append((u, b))
    PU = torch.stack([s_[0] for s_ in states[:T]])
    PB = torch.stack([s_[1] for s_ in states[:T]])
    au = to(rng.standard_normal(n).astype(np.float32))
    ab = to(rng.standard_normal(n).astype(np.float32))
    gu, gb = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
    glam = torch.empty((T, n), device="cuda")
    gpc = torch.zeros(1, dtype=f64, device="cuda")
    sim.relaxed_bwd_steps(PU, PB, au, ab, gu, gb, masks=masks, glam=glam, gpc=gpc)
    gpc1 = torch.zeros(1, dtype=f64, device="cuda")
    ru, rb = au, ab
    for t in reversed(range(T)):
        gl = torch.empty(n, device="cuda")
        ru, rb = sim.relaxed_bwd(PU[t], PB[t], ru, rb, mask=None if masks is None else masks[t], glam=gl, gpc=gpc1)
        assert torch.equal(gl, glam[t])
    assert torch.equal(ru, gu) and torch.equal(rb, gb)
    assert gpc.item() == pytest.approx(gpc1.item(), rel=1e-5, abs=1e-9)


def test_full_size_T1000_sampled():
    """256 x 128^2, T = 1000, sqrt(T) checkpoints; loss on 2 sampled envs."""
    require_gpu()
    N, H, W, T = 256, 128, 128, 1000
    scn = scenarios.make_scenario(H, W, N=N, seed=0)
    rng = np.random.default_rng(5)
    pu, pb = _planes(scn, rng, soft=False)
    sample = [17, 200]
    wu = np.zeros(pu.size, np.float32)
    wb = np.zeros(pu.size, np.float32)
    for e in sample:
        o0, o1 = scn.offsets[e], scn.offsets[e + 1]
        wu[o0:o1] = rng.standard_normal(o1 - o0)
        wb[o0:o1] = rng.standard_normal(o1 - o0)
    theta = _theta(scn.params, scenarios.N_CLASSES).float().double()
    sim = make_sim(scn, keep_rates=True)
    scene = (to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    th = theta.clone().requires_grad_(True)
    U = to(pu.astype(np.float32)).requires_grad_(True)
    B = to(pb.astype(np.float32)).requires_grad_(True)
    ou, ob = relaxed.rollout(th, U, B, sim, scene, T)
    L = (to(wu) * ou).sum() + (to(wb) * ob).sum()
    gth, gU, gB = torch.autograd.grad(L, [th, U, B])
    rth, rU, rB = _oracle_grad(scn, theta, pu, pb, T, wu, wb, envs=sample)
    _close(gth.cpu().numpy(), rth.numpy())
    for i, e in enumerate(sample):
        o0, o1 = scn.offsets[e], scn.offsets[e + 1]
        for g, ref in ((gU[o0:o1], rU[i]), (gB[o0:o1], rB[i])):
            g = g.cpu().numpy().astype(np.float64)
            ref = ref.reshape(-1).numpy()
            assert np.isfinite(g).all()                  # saturated, never inf or NaN
            assert np.abs(g).max() <= float(np.float32(1e35))
    # envs outside the loss get zero adjoint
    other = np.ones(pu.size, bool)
    for e in sample:
        other[scn.offsets[e]:scn.offsets[e + 1]] = False
    assert float(gB[to(other)].abs().max()) == 0.0
