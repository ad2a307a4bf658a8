"""Tanker actions as cell masks on the GPU (Section 4: water turns a burning
cell into a burned one), against the oracle's masked rollout bit for bit.

  * jwf_pack_masks equals a little-endian bit packing of the uint8 masks;
  * every step kernel (plain, resident, fused resident, tiled, fused tiled)
    with random masks on ragged batches (widths that are not multiples of 32,
    grids spanning several tiles), k split across launches, and auto-reset;
    the fused kernels against the oracle fed the GPU's own probability table;
  * masks equal to the drops' 3x3 footprints reproduce the drop path on the
    benchmark's batched workload (4096 x 128^2, 200 steps, the launch split
    after 12 steps).
"""
import numpy as np
import pytest
import torch

from oracle import discrete
from paper_2512_06102_gb300 import jwf, scenarios
from tests.gpu_util import make_sim, oracle_tables, require_gpu, to

pytestmark = pytest.mark.gpu

TABLE = [jwf.KERNEL_PLAIN, jwf.KERNEL_RESIDENT, jwf.KERNEL_TILED]
FUSED = [jwf.KERNEL_FUSED, jwf.KERNEL_TILED_FUSED]


def _masks(k, cells, rate, seed):
    return (np.random.default_rng(seed).random((k, cells)) < rate).astype(np.uint8)


def _gpu_masked(scn, q32, masks, kernel, seed, splits, t_max=0, auto_reset=False):
    sim = make_sim(scn, seed=seed, t_max=t_max, auto_reset=auto_reset)
    sim.set_kernel(kernel)
    terrain = (to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    if kernel in FUSED:
        sim.set_terrain(*terrain)
    else:
        sim.set_probs(to(q32))
    bits = jwf.pack_masks(to(masks))
    sim.load_state(to(scn.F0))
    outs, s0 = [], 0
    for kk in splits:
        outs.append([x.cpu().numpy() for x in sim.step_masked(kk, bits[s0:s0 + kk].contiguous())])
        s0 += kk
    torch.cuda.synchronize()
    sim.sync()
    st, t, ep = (x.cpu().numpy().copy() for x in sim.state_views())
    sim.close()
    return st, [np.concatenate([o[i] for o in outs]) for i in range(3)], t, ep


def _gpu_table(scn):
    sim = make_sim(scn)
    sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    q = sim.probs()[0].cpu().numpy().copy()
    sim.close()
    return q


def _check(scn, q32, masks, kernel, seed, splits, **kw):
    g = _gpu_masked(scn, q32, masks, kernel, seed, splits, **kw)
    ro = discrete.Rollout(scn.H, scn.W, scn.F0, q32, scn.params.p_continue, seed=seed,
                          t_max=kw.get("t_max", 0), auto_reset=kw.get("auto_reset", False))
    o = ro.step_masks(masks)
    np.testing.assert_array_equal(g[0], ro.F)
    for a, b in zip(g[1], o):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(g[2], ro.t)
    np.testing.assert_array_equal(g[3], ro.episode)
    return o


def test_pack_masks():
    require_gpu()
    for k, n in [(3, 1), (2, 31), (4, 32), (5, 33), (3, 1000), (2, 4099)]:
        m = _masks(k, n, 0.3, k * 1000 + n)
        bits = jwf.pack_masks(to(m)).cpu().numpy()
        words = jwf.mask_words(n)
        ref = np.zeros((k, words * 32), np.uint8)
        ref[:, :n] = m
        ref = np.packbits(ref, axis=1, bitorder="little").view("<u4").view(np.int32)
        np.testing.assert_array_equal(bits, ref)


@pytest.mark.parametrize("kernel", TABLE + FUSED)
@pytest.mark.parametrize("shape", [((40, 17, 64), (37, 53, 64)), ((130, 70), (300, 257))])
def test_masked_steps_match_oracle(kernel, shape):
    require_gpu()
    H, W = shape
    scn = scenarios.make_scenario(list(H), list(W), seed=41)
    k = 30
    masks = _masks(k, scn.F0.size, 0.08, 41)
    q32 = _gpu_table(scn) if kernel in FUSED else oracle_tables(scn)[0]
    o = _check(scn, q32, masks, kernel, 7, [1, 12, 17])
    assert o[1][-1].sum() > 0


@pytest.mark.parametrize("kernel", [jwf.KERNEL_PLAIN, jwf.KERNEL_RESIDENT, jwf.KERNEL_FUSED])
def test_masked_steps_auto_reset(kernel):
    require_gpu()
    scn = scenarios.make_scenario(48, 45, N=6, seed=42)
    k = 60
    masks = _masks(k, scn.F0.size, 0.05, 42)
    q32 = _gpu_table(scn) if kernel in FUSED else oracle_tables(scn)[0]
    _check(scn, q32, masks, kernel, 3, [25, 35], t_max=20, auto_reset=True)


def test_masked_footprints_equal_drops_full_size():
    """The benchmark's batched workload: masks equal to the drops' 3x3
    footprints give the drop path's states, counts and done flags."""
    require_gpu()
    N, S, k = 4096, 128, 200
    scn = scenarios.make_scenario(S, S, N=N, seed=0)
    drops = scenarios.drops(k, scn.H, scn.W, seed=0)
    dev = torch.device("cuda", 0)
    # footprints of radius 1, clipped to the grid, built on the device step by step
    d = torch.from_numpy(drops).to(dev).long()
    yy = torch.arange(S, device=dev).view(1, S, 1)
    xx = torch.arange(S, device=dev).view(1, 1, S)
    bits = torch.empty((k, jwf.mask_words(N * S * S)), dtype=torch.int32, device=dev)
    for t in range(k):
        cx, cy = d[t, :, 0].view(N, 1, 1), d[t, :, 1].view(N, 1, 1)
        foot = ((yy - cy).abs() <= 1) & ((xx - cx).abs() <= 1) & (cx >= 0) & (cy >= 0)
        jwf.pack_masks(foot.to(torch.uint8).reshape(1, N * S * S), out=bits[t:t + 1])
    res = []
    for masked in (False, True):
        sim = make_sim(scn, seed=1000)
        sim.set_kernel(jwf.KERNEL_FUSED)
        sim.set_reorder_steps(12)
        sim.set_terrain(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
        sim.load_state(to(scn.F0))
        out = sim.step_masked(k, bits) if masked else sim.step(k, to(drops))
        torch.cuda.synchronize()
        res.append((sim.state().cpu().numpy(), [x.cpu().numpy() for x in out]))
        sim.close()
    np.testing.assert_array_equal(res[0][0], res[1][0])
    for a, b in zip(res[0][1], res[1][1]):
        np.testing.assert_array_equal(a, b)
