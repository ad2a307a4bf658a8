"""Trajectory recording and the straight-through rollout on the GPU.

  * jwf_step_record's history equals the states of the same run stepped one
    step at a time, for the plain, resident (table and fused) and tiled
    kernels, with drops (and with auto-reset where the kernel supports it);
  * with the oracle's FP32 table, the recorded trajectory equals the C
    oracle's, step by step;
  * the straight-through gradient (stochastic forward, relaxed adjoint along
    the sampled trajectory) equals the FP64 oracle's chain of relaxed-step
    adjoints linearised at the same hard states, within 1e-4 relative.
"""
import numpy as np
import pytest
import torch

from oracle import discrete, prob
from oracle import relaxed as orelaxed
from paper_2512_06102_gb300 import jwf, relaxed, scenarios
from tests.gpu_util import make_sim, oracle_tables, require_gpu, to

pytestmark = pytest.mark.gpu
f64 = torch.float64


def _run(scn, k, drops, kernel, record, seed=5, **kw):
    sim = make_sim(scn, seed=seed, **kw)
    sim.set_terrain(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    if kernel in (jwf.KERNEL_PLAIN, jwf.KERNEL_RESIDENT, jwf.KERNEL_TILED):
        sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    sim.set_kernel(kernel)
    sim.load_state(to(scn.F0))
    dr = None if drops is None else to(drops)
    if record:
        hist = torch.zeros((k, sim.cells), dtype=torch.uint8, device="cuda")
        out = sim.step(k, dr, history=hist)
        res = hist.cpu().numpy(), [x.cpu().numpy() for x in out]
    else:
        rows, outs = [], []
        for t in range(k):
            outs.append(sim.step(1, None if dr is None else dr[t:t + 1]))
            rows.append(sim.state())
        res = torch.stack(rows).cpu().numpy(), [torch.cat([o[i] for o in outs]).cpu().numpy() for i in range(3)]
    sim.close()
    return res


@pytest.mark.parametrize("kernel,shape,N,kw", [
    (jwf.KERNEL_PLAIN, (37, 45), 5, {"auto_reset": True, "t_max": 9}),
    (jwf.KERNEL_RESIDENT, (37, 45), 5, {"auto_reset": True, "t_max": 9}),
    (jwf.KERNEL_FUSED, (64, 64), 7, {}),
    (jwf.KERNEL_FUSED, (33, 20), 6, {"auto_reset": True, "t_max": 5}),
    (jwf.KERNEL_TILED_FUSED, (150, 300), 2, {}),
])
def test_history_equals_single_steps(kernel, shape, N, kw):
    require_gpu()
    k = 22
    scn = scenarios.make_scenario(shape[0], shape[1], N=N, seed=41)
    drops = scenarios.drops(k, scn.H, scn.W, seed=4)
    a = _run(scn, k, drops, kernel, True, **kw)
    b = _run(scn, k, drops, kernel, False, **kw)
    np.testing.assert_array_equal(a[0], b[0])
    for x, y in zip(a[1], b[1]):
        np.testing.assert_array_equal(x, y)


def test_history_equals_oracle_trajectory():
    require_gpu()
    k = 18
    scn = scenarios.make_scenario(30, 26, N=4, seed=42)
    drops = scenarios.drops(k, scn.H, scn.W, seed=5)
    q32 = oracle_tables(scn)[0]
    sim = make_sim(scn, seed=6)
    sim.set_probs(to(q32))
    sim.set_kernel(jwf.KERNEL_RESIDENT)
    sim.load_state(to(scn.F0))
    hist = torch.zeros((k, sim.cells), dtype=torch.uint8, device="cuda")
    sim.step(k, to(drops), history=hist)
    h = hist.cpu().numpy()
    sim.close()
    ro = discrete.Rollout(scn.H, scn.W, scn.F0, q32, scn.params.p_continue, seed=6)
    for t in range(k):
        ro.step(1, np.ascontiguousarray(drops[t:t + 1]))
        np.testing.assert_array_equal(h[t], ro.F)


def _close(g, ref, rel=1e-4, floor=1e-7):
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    tol = rel * np.abs(ref) + floor * np.abs(ref).max()
    bad = np.abs(g - ref) > tol
    assert not bad.any(), f"{bad.sum()} off; worst {np.max(np.abs(g - ref) / np.maximum(np.abs(ref), 1e-300))}"


def test_straight_through_matches_oracle():
    require_gpu()
    H, W, N, T = 40, 44, 3, 15
    scn = scenarios.make_scenario(H, W, N=N, seed=43)
    C = scenarios.N_CLASSES
    q32, r32, _, _ = oracle_tables(scn)
    p = scn.params
    theta = torch.tensor([p.p_base, p.alpha_w1, p.alpha_w2, p.alpha_s, p.alpha_gamma, p.p_continue]
                         + list(p.mu_veg) + list(p.mu_den), dtype=f64).float().double()
    sim = make_sim(scn, seed=8, keep_rates=True)
    sim.set_probs(to(q32), to(r32))
    sim.set_kernel(jwf.KERNEL_RESIDENT)
    scene = (to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    rng = np.random.default_rng(8)
    wu = rng.standard_normal(N * H * W).astype(np.float32)
    wb = rng.standard_normal(N * H * W).astype(np.float32)
    th = theta.clone().requires_grad_(True)
    ou, ob = relaxed.straight_through(th, sim, scene, to(scn.F0), T, build_tables=False)
    L = (to(wu) * ou).sum() + (to(wb) * ob).sum()
    (g,) = torch.autograd.grad(L, [th])
    sim.close()
    # the oracle's trajectory with the same table and seed
    ro = discrete.Rollout(scn.H, scn.W, scn.F0, q32, p.p_continue, seed=8)
    states = []
    for t in range(T):
        states.append(ro.F.copy().reshape(N, H, W))
        ro.step(1)
    fin = ro.F.reshape(N, H, W)
    np.testing.assert_array_equal(ou.detach().cpu().numpy().reshape(N, H, W), (fin <= 1).astype(np.float32))
    cls = torch.as_tensor(scn.cls.reshape(N, H, W)).long()
    dem = torch.as_tensor(scn.dem.reshape(N, H, W).astype(np.float64))

    def r_of(t_):
        return prob.rates(cls, dem, torch.as_tensor(scn.wind_speed.astype(np.float64)),
                          torch.as_tensor(scn.wind_dir.astype(np.float64)), t_[0], t_[1], t_[2], t_[3], t_[4],
                          t_[6:6 + C], t_[6 + C:6 + 2 * C], p.cell_size)

    ref = orelaxed.straight_through_grad(states, r_of, theta, torch.as_tensor(wu.astype(np.float64)).reshape(N, H, W),
                                         torch.as_tensor(wb.astype(np.float64)).reshape(N, H, W))
    _close(g.cpu().numpy(), ref.numpy())
    assert np.abs(ref.numpy()).max() > 0
