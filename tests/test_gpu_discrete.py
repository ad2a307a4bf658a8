"""Discrete step on the GPU against the CPU oracle: bit-exact states, counts and
done flags, for both step kernels, given the same float table (computed by the
FP64 oracle and rounded) and the same Philox stream.

Kernels: plain (one launch per step), resident (whole env in shared memory,
k steps per launch), tiled (128 x 256 tiles with halos, up to 16 steps per
launch, cold tiles skipped), and the fused variants of the last two, which
evaluate probabilities from the terrain and must equal the table path.

Edge cases: single grid of the plain workload (64x64, 100 steps), the batched
workload at reduced and full size (sampled), ragged batches, widths that are
not multiples of 32 (1, 17, 33, 37), one-row and one-cell grids, no fuel at
all, every cell burning, probability 0 and 1 (Chebyshev square), auto-reset
with an episode limit, direct masks and resets, and k split across launches.
"""
import numpy as np
import pytest
import torch

from oracle import discrete
from paper_2512_06102_gb300 import jwf, scenarios
from tests.gpu_util import make_sim, oracle_tables, require_gpu, to

pytestmark = pytest.mark.gpu
KERNELS = [jwf.KERNEL_PLAIN, jwf.KERNEL_RESIDENT, jwf.KERNEL_TILED]


def _run_both(scn, q32, k, drops=None, seed=0, kernel=jwf.KERNEL_AUTO, t_max=0, auto_reset=False,
              splits=None, threads=0, tile_copy=None):
    sim = make_sim(scn, seed=seed, t_max=t_max, auto_reset=auto_reset)
    sim.set_kernel(kernel, threads)
    if tile_copy is not None:
        sim.set_tile_copy(tile_copy)
        assert sim.tile_copy() == tile_copy
    sim.set_probs(to(q32))
    sim.load_state(to(scn.F0))
    ro = discrete.Rollout(scn.H, scn.W, scn.F0, q32, scn.params.p_continue, seed=seed, t_max=t_max,
                          auto_reset=auto_reset)
    splits = splits or [k]
    outs_g, outs_o = [], []
    s0 = 0
    for kk in splits:
        dr = None if drops is None else drops[s0:s0 + kk]
        g = sim.step(kk, drops=None if dr is None else to(dr))
        o = ro.step(kk, dr)
        outs_g.append([x.cpu().numpy() for x in g])
        outs_o.append(o)
        s0 += kk
    torch.cuda.synchronize()
    sim.sync()
    state = sim.state().cpu().numpy()
    _, t, ep = sim.state_views()
    np.testing.assert_array_equal(state, ro.F)
    for g, o in zip(outs_g, outs_o):
        for a, b in zip(g, o):
            np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(t.cpu().numpy(), ro.t)
    np.testing.assert_array_equal(ep.cpu().numpy(), ro.episode)
    sim.close()
    return ro


@pytest.mark.parametrize("kernel", KERNELS)
def test_plain_single_env(kernel):
    require_gpu()
    scn = scenarios.plain_single_env(64, 64)
    q32 = oracle_tables(scn)[0]
    ro = _run_both(scn, q32, 100, seed=0, kernel=kernel)
    assert (ro.F == 3).sum() > 100          # the fire did spread


@pytest.mark.parametrize("kernel", KERNELS)
def test_batched_with_drops(kernel):
    require_gpu()
    scn = scenarios.make_scenario(128, 128, N=24, seed=0)
    q32 = oracle_tables(scn)[0]
    drops = scenarios.drops(200, scn.H, scn.W, seed=0)
    _run_both(scn, q32, 200, drops=drops, seed=0, kernel=kernel)


@pytest.mark.parametrize("threads", [32, 64, 128, 256, 512, 1024])
def test_resident_thread_counts(threads):
    require_gpu()
    scn = scenarios.make_scenario(96, 80, N=5, seed=9)
    q32 = oracle_tables(scn)[0]
    drops = scenarios.drops(60, scn.H, scn.W, seed=9)
    _run_both(scn, q32, 60, drops=drops, seed=4, kernel=jwf.KERNEL_RESIDENT, threads=threads)


@pytest.mark.parametrize("kernel", KERNELS)
def test_ragged_batch(kernel):
    require_gpu()
    sides = scenarios.ragged_sides(16, 32, 512, seed=4)
    scn = scenarios.make_scenario(sides, sides, seed=4)
    q32 = oracle_tables(scn)[0]
    drops = scenarios.drops(40, scn.H, scn.W, seed=4)
    _run_both(scn, q32, 40, drops=drops, seed=7, kernel=kernel)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("shape", [(5, 1), (1, 17), (33, 33), (20, 37), (1, 1), (64, 97)])
def test_odd_shapes(kernel, shape):
    require_gpu()
    H, W = shape
    scn = scenarios.make_scenario(H, W, N=3, seed=11)
    q32 = oracle_tables(scn)[0]
    drops = scenarios.drops(30, scn.H, scn.W, seed=11)
    _run_both(scn, q32, 30, drops=drops, seed=2, kernel=kernel)


@pytest.mark.parametrize("kernel", KERNELS)
def test_degenerate_grids(kernel):
    require_gpu()
    H = W = 40
    scn = scenarios.make_scenario(H, W, N=4, seed=2)
    F0 = scn.F0.reshape(4, H, W).copy()
    F0[0] = 0                   # no fuel anywhere
    F0[1] = 2                   # everything burning
    F0[2] = 3                   # everything burned
    F0[3, :, :] = 1
    F0[3, 0, 0] = 2             # a corner fire
    scn.F0 = F0.reshape(-1)
    q32 = oracle_tables(scn)[0]
    _run_both(scn, q32, 25, seed=1, kernel=kernel)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("qval", [0.0, 1.0])
def test_extreme_probabilities(kernel, qval):
    require_gpu()
    H = W = 65
    scn = scenarios.plain_single_env(H, W)
    q32 = np.full((H * W, 8), qval, np.float32)
    ro = _run_both(scn, q32, 20, seed=0, kernel=kernel)
    if qval == 1.0:
        y, x = np.mgrid[0:H, 0:W]
        cheb = np.maximum(abs(y - H // 2), abs(x - W // 2)) <= 20
        np.testing.assert_array_equal(((ro.F == 2) | (ro.F == 3)).reshape(H, W), cheb)


@pytest.mark.parametrize("kernel", KERNELS)
def test_auto_reset_episode_limit(kernel):
    require_gpu()
    scn = scenarios.make_scenario(48, 48, N=10, seed=6)
    q32 = oracle_tables(scn)[0]
    drops = scenarios.drops(90, scn.H, scn.W, seed=6)
    ro = _run_both(scn, q32, 90, drops=drops, seed=3, kernel=kernel, t_max=25, auto_reset=True)
    assert (ro.episode >= 3).all()


@pytest.mark.parametrize("kernel", KERNELS)
def test_k_split_across_launches(kernel):
    require_gpu()
    scn = scenarios.make_scenario(64, 64, N=6, seed=8)
    q32 = oracle_tables(scn)[0]
    drops = scenarios.drops(50, scn.H, scn.W, seed=8)
    _run_both(scn, q32, 50, drops=drops, seed=5, kernel=kernel, splits=[1, 7, 20, 22])


def test_action_and_reset_api():
    require_gpu()
    scn = scenarios.make_scenario(32, 48, N=3, seed=1)
    q32 = oracle_tables(scn)[0]
    sim = make_sim(scn, seed=2)
    sim.set_probs(to(q32))
    sim.load_state(to(scn.F0))
    sim.step(5)
    before = sim.state().cpu().numpy()
    mask = (np.random.default_rng(0).random(before.size) < 0.5).astype(np.uint8)
    sim.apply_action(to(mask))
    after = sim.state().cpu().numpy()
    want = np.where((before == 2) & (mask == 1), 3, before)
    np.testing.assert_array_equal(after, want)
    sim.reset(to(np.array([0, 1, 0], np.uint8)))
    s, t, ep = (x.cpu().numpy() for x in sim.state_views())
    o1, o2 = scn.offsets[1], scn.offsets[2]
    np.testing.assert_array_equal(s[o1:o2], scn.F0[o1:o2])
    np.testing.assert_array_equal(s[:o1], after[:o1])
    assert t.tolist() == [5, 0, 5] and ep.tolist() == [0, 1, 0]
    sim.close()


def test_full_size_resident_sampled():
    """4096 x 128^2, 200 steps with drops, in the benchmark's launch
    configuration (resident kernel, one launch); oracle on a sample of envs."""
    require_gpu()
    from oracle import prob
    N, H, W, k = 4096, 128, 128, 200
    scn = scenarios.make_scenario(H, W, N=N, seed=0)
    sim = make_sim(scn, seed=0)
    sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    q_gpu = sim.probs()[0]
    rng = np.random.default_rng(2)
    sample = sorted(set(rng.choice(N, 6, replace=False).tolist() + [0, N - 1]))
    p = scn.params.as_dict()
    q_s = []
    for e in sample:
        q32, _, _, _ = prob.table_f32(scn.env(e, scn.cls)[None], scn.env(e, scn.dem)[None],
                                      scn.wind_speed[e:e + 1], scn.wind_dir[e:e + 1], p, 30.0)
        q_s.append(q32.reshape(-1, 8))
    # the step draws against the GPU table; use the oracle's rounding of it
    # only where the two agree bit for bit (they are within 1e-6 relative)
    q_full = q_gpu.clone()
    for e, qe in zip(sample, q_s):
        q_full[scn.offsets[e]:scn.offsets[e + 1]] = to(qe)
    sim.set_probs(q_full)
    sim.load_state(to(scn.F0))
    drops = scenarios.drops(k, scn.H, scn.W, seed=0)
    b, d, done = sim.step(k, drops=to(drops))
    torch.cuda.synchronize()
    state = sim.state().cpu().numpy()
    b, d, done = b.cpu().numpy(), d.cpu().numpy(), done.cpu().numpy()
    Hs, Ws = np.full(len(sample), H, np.int32), np.full(len(sample), W, np.int32)
    F0s = np.concatenate([scn.env(e, scn.F0).reshape(-1) for e in sample])
    ro = discrete.Rollout(Hs, Ws, F0s, np.concatenate(q_s), scn.params.p_continue, seed=0,
                          env_ids=np.array(sample, np.int32))
    ob, od, odone = ro.step(k, np.ascontiguousarray(drops[:, sample]))
    for i, e in enumerate(sample):
        np.testing.assert_array_equal(state[scn.offsets[e]:scn.offsets[e + 1]], ro.env_state(i).reshape(-1))
    np.testing.assert_array_equal(b[:, sample], ob)
    np.testing.assert_array_equal(d[:, sample], od)
    np.testing.assert_array_equal(done[:, sample], odone)
    # properties that hold for every env
    assert ((state == 0) == (scn.F0 == 0)).all()          # no-fuel never changes
    assert (b[-1] >= 0).all() and ((done[-1] == 1) | (b[-1] > 0)).all()
    sim.close()


def test_plain_and_resident_agree_full_size():
    require_gpu()
    N, H, W, k = 4096, 128, 128, 60
    scn = scenarios.make_scenario(H, W, N=N, seed=3)
    drops = to(scenarios.drops(k, scn.H, scn.W, seed=3))
    res = []
    for kernel in KERNELS:
        sim = make_sim(scn, seed=1)
        sim.set_kernel(kernel)
        sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
        sim.load_state(to(scn.F0))
        out = sim.step(k, drops=drops)
        torch.cuda.synchronize()
        res.append((sim.state().cpu().numpy(), [x.cpu().numpy() for x in out]))
        sim.close()
    np.testing.assert_array_equal(res[0][0], res[1][0])
    for a, b in zip(res[0][1], res[1][1]):
        np.testing.assert_array_equal(a, b)


# ---------------------------------------------------------------------------
# fused step: probabilities evaluated on the spot from the terrain, with the
# same rate code as the table kernel, so its trajectories equal the table
# path's bit for bit (the table path equals the oracle given the same table,
# and the table kernel is within 1e-6 of the FP64 oracle)
# ---------------------------------------------------------------------------
def _gpu_run(scn, k, drops, kernel, seed, threads=0, t_max=0, auto_reset=False):
    sim = make_sim(scn, seed=seed, t_max=t_max, auto_reset=auto_reset)
    sim.set_kernel(kernel, threads)
    terrain = (to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    if kernel == jwf.KERNEL_FUSED:
        sim.set_terrain(*terrain)
    else:
        sim.precompute_probs(*terrain)
    sim.load_state(to(scn.F0))
    out = sim.step(k, drops=None if drops is None else to(drops))
    torch.cuda.synchronize()
    sim.sync()
    s, t, ep = (x.cpu().numpy().copy() for x in sim.state_views())
    res = (s, [x.cpu().numpy() for x in out], t, ep)
    sim.close()
    return res


def _same(a, b):
    np.testing.assert_array_equal(a[0], b[0])
    for x, y in zip(a[1], b[1]):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a[2], b[2])
    np.testing.assert_array_equal(a[3], b[3])


@pytest.mark.parametrize("threads", [0, 32, 256])
@pytest.mark.parametrize("shape,N", [((128, 128), 16), ((37, 45), 5), ((1, 17), 3), ((300, 260), 2)])
def test_fused_equals_table_path(shape, N, threads):
    require_gpu()
    H, W = shape
    scn = scenarios.make_scenario(H, W, N=N, seed=21)
    k = 80
    drops = scenarios.drops(k, scn.H, scn.W, seed=21)
    a = _gpu_run(scn, k, drops, jwf.KERNEL_RESIDENT, 5, threads)
    b = _gpu_run(scn, k, drops, jwf.KERNEL_FUSED, 5, threads)
    _same(a, b)
    assert (a[0] == 3).sum() > 0 or H * W < 64


def test_fused_ragged_auto_reset_equals_plain():
    require_gpu()
    sides = scenarios.ragged_sides(12, 32, 512, seed=6)
    scn = scenarios.make_scenario(sides, sides[::-1], seed=6)
    k = 70
    drops = scenarios.drops(k, scn.H, scn.W, seed=6)
    a = _gpu_run(scn, k, drops, jwf.KERNEL_PLAIN, 9, t_max=30, auto_reset=True)
    b = _gpu_run(scn, k, drops, jwf.KERNEL_FUSED, 9, t_max=30, auto_reset=True)
    _same(a, b)
    assert (b[3] >= 2).all()


def test_fused_equals_table_path_full_size():
    """4096 x 128^2, one 200-step episode with drops (the benchmark workload)."""
    require_gpu()
    scn = scenarios.make_scenario(128, 128, N=4096, seed=0)
    drops = scenarios.drops(200, scn.H, scn.W, seed=0)
    a = _gpu_run(scn, 200, drops, jwf.KERNEL_RESIDENT, 1000)
    b = _gpu_run(scn, 200, drops, jwf.KERNEL_FUSED, 1000)
    _same(a, b)


# ---------------------------------------------------------------------------
# tiled path on grids spanning several tiles
# ---------------------------------------------------------------------------
def _fire_drops(scn, k, seed):
    """Drops aimed at the initial fires (so that they douse burning cells on
    tile borders and corners), one per env and step, jittered by +-2 cells."""
    rng = np.random.default_rng(seed)
    out = np.full((k, scn.N, 2), -1, np.int32)
    for e in range(scn.N):
        F = scn.env(e, scn.F0)
        ys, xs = np.nonzero(F == 2)
        for s in range(k):
            if len(ys) and rng.random() < 0.7:
                j = rng.integers(len(ys))
                out[s, e] = (xs[j] + rng.integers(-2, 3), ys[j] + rng.integers(-2, 3))
            elif rng.random() < 0.5:
                out[s, e] = (rng.integers(0, scn.W[e]), rng.integers(0, scn.H[e]))
    return out


def _fires_on_tile_corners(scn):
    """Add fires at tile corners and edges (rows 127/128, columns 255/256)."""
    for e in range(scn.N):
        F = scn.env(e, scn.F0)
        H, W = F.shape
        for y, x in [(127, 255), (128, 256), (127, 256), (128, 255), (0, W - 1), (H - 1, 0), (64, 256)]:
            if y < H and x < W:
                F[y, x] = 2


@pytest.mark.parametrize("shape,N,k", [((300, 700), 2, 37), ((129, 257), 3, 50), ((520, 300), 1, 33)])
def test_tiled_multi_tile_matches_oracle(shape, N, k):
    require_gpu()
    H, W = shape
    scn = scenarios.make_scenario(H, W, N=N, seed=31)
    _fires_on_tile_corners(scn)
    q32 = oracle_tables(scn)[0]
    drops = _fire_drops(scn, k, 31)
    _run_both(scn, q32, k, drops=drops, seed=8, kernel=jwf.KERNEL_TILED, splits=[k // 2, k - k // 2])


@pytest.mark.parametrize("tma", [True, False])
@pytest.mark.parametrize("shapes", [[(320, 640), (200, 336)],                  # every env takes the tensor copy
                                    [(200, 336), (150, 300), (96, 160)]])     # a mix: rows of 300, odd offsets
def test_tiled_tma_and_loads_match_oracle(shapes, tma):
    """The tiled step with its regions staged by TMA tensor copies (envs whose
    first cell and row pitch are 16-byte multiples; quiet tiles copied by a
    tensor load and store) and by plain loads equals the oracle."""
    require_gpu()
    H = [s[0] for s in shapes]
    W = [s[1] for s in shapes]
    scn = scenarios.make_scenario(H, W, seed=33)
    _fires_on_tile_corners(scn)
    q32 = oracle_tables(scn)[0]
    k = 40
    drops = _fire_drops(scn, k, 33)
    _run_both(scn, q32, k, drops=drops, seed=9, kernel=jwf.KERNEL_TILED, splits=[7, 16, 17], tile_copy=tma)


def test_tiled_fused_equals_tiled_table():
    require_gpu()
    scn = scenarios.make_scenario(600, 900, N=2, seed=32)
    _fires_on_tile_corners(scn)
    k = 60
    drops = _fire_drops(scn, k, 32)
    a = _gpu_run(scn, k, drops, jwf.KERNEL_TILED, 3)
    b = _gpu_run(scn, k, drops, jwf.KERNEL_TILED_FUSED, 3)
    c = _gpu_run(scn, k, drops, jwf.KERNEL_PLAIN, 3)
    _same(a, b)
    _same(a, c)


def test_tiled_large_grids_sampled():
    """8 x 4096^2 (the large-map workload) for 48 steps with drops: tiled fused
    against the plain path on all grids, and the oracle on one grid."""
    require_gpu()
    from oracle import prob
    N, H, W, k = 8, 4096, 4096, 48
    scn = scenarios.make_scenario(H, W, N=N, seed=0)
    drops = _fire_drops(scn, k, 0)
    a = _gpu_run(scn, k, drops, jwf.KERNEL_TILED_FUSED, 11)
    b = _gpu_run(scn, k, drops, jwf.KERNEL_PLAIN, 11)
    _same(a, b)
    # the oracle on grid 5 with the GPU's own table for that grid replaced by the oracle's
    e = 5
    q32, _, _, _ = prob.table_f32(scn.env(e, scn.cls)[None], scn.env(e, scn.dem)[None],
                                  scn.wind_speed[e:e + 1], scn.wind_dir[e:e + 1], scn.params.as_dict(), 30.0)
    sim = make_sim(scn, seed=11)
    sim.set_kernel(jwf.KERNEL_TILED)
    sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    qg = sim.probs()[0]
    qg[scn.offsets[e]:scn.offsets[e + 1]] = to(q32.reshape(-1, 8))
    sim.load_state(to(scn.F0))
    out = sim.step(k, drops=to(drops))
    torch.cuda.synchronize()
    st = sim.state()[scn.offsets[e]:scn.offsets[e + 1]].cpu().numpy()
    ro = discrete.Rollout([H], [W], scn.env(e, scn.F0).reshape(-1), q32.reshape(-1, 8), scn.params.p_continue,
                          seed=11, env_ids=[e])
    ob, od, odone = ro.step(k, np.ascontiguousarray(drops[:, e:e + 1]))
    np.testing.assert_array_equal(st, ro.F)
    np.testing.assert_array_equal(out[0].cpu().numpy()[:, e:e + 1], ob)
    np.testing.assert_array_equal(out[1].cpu().numpy()[:, e:e + 1], od)
    sim.close()


def test_tiled_copy_wait_runs_out_and_context_recovers():
    """The tiled kernels' wait for a tensor copy is bounded: with the
    diagnostic that arms the wait but issues no copy, every wait runs out
    after 1 ms, the kernel leaves its tile and sets the status word, and
    jwf_sync reports JWF_ETIMEOUT (no fault, no hang).  Afterwards the same
    context, reloaded, steps exactly like the oracle."""
    require_gpu()
    scn = scenarios.make_scenario(128, 256, N=1, seed=34)
    _fires_on_tile_corners(scn)
    q32 = oracle_tables(scn)[0]
    sim = make_sim(scn, seed=4)
    sim.set_kernel(jwf.KERNEL_TILED)
    sim.set_probs(to(q32))
    assert sim.tile_copy()
    sim.load_state(to(scn.F0))
    sim.set_tile_copy_wait(1_000_000, no_copy=True)
    sim.step(3)
    with pytest.raises(jwf.JwfError) as err:
        sim.sync()
    assert err.value.status == 4          # JWF_ETIMEOUT
    sim.set_tile_copy_wait()              # 2 s, copies issued
    sim.sync()                            # the status word was cleared by the report
    k = 20
    sim.load_state(to(scn.F0))
    out = sim.step(k)
    torch.cuda.synchronize()
    sim.sync()
    ro = discrete.Rollout(scn.H, scn.W, scn.F0, q32, scn.params.p_continue, seed=4)
    ob, od, odone = ro.step(k)
    np.testing.assert_array_equal(sim.state().cpu().numpy(), ro.F)
    np.testing.assert_array_equal(out[0].cpu().numpy(), ob)
    sim.close()


@pytest.mark.parametrize("threads", [0, 1024])
@pytest.mark.parametrize("kernel", [jwf.KERNEL_RESIDENT, jwf.KERNEL_FUSED])
def test_resident_maximum_size(kernel, threads):
    """The largest grids the resident kernels hold in shared memory (longer
    side 512, the top size class; 512 x 500 leaves a partial word in every
    row) next to a small one, with drops, against the oracle bit for bit; by
    default and with 1024 threads a grid (the largest block whose warp
    scratch still fits beside the grid)."""
    require_gpu()
    H = [512, 512, 33]
    W = [512, 500, 512]
    scn = scenarios.make_scenario(H, W, seed=35)
    _fires_on_tile_corners(scn)
    q32 = oracle_tables(scn)[0]
    k = 30
    drops = _fire_drops(scn, k, 35)
    sim = make_sim(scn, seed=6)
    sim.set_kernel(kernel, threads)
    if kernel == jwf.KERNEL_FUSED:
        sim.set_terrain(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
        fused = sim
        # the fused rates equal the oracle's table only to 1e-6: compare with the table path instead
        ref = make_sim(scn, seed=6)
        ref.set_kernel(jwf.KERNEL_RESIDENT)
        ref.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
        outs = []
        for s in (fused, ref):
            s.load_state(to(scn.F0))
            o = [x.cpu().numpy() for x in s.step(k, to(drops))]
            outs.append((s.state().cpu().numpy(), o))
            s.close()
        np.testing.assert_array_equal(outs[0][0], outs[1][0])
        for a, b in zip(outs[0][1], outs[1][1]):
            np.testing.assert_array_equal(a, b)
        return
    sim.set_probs(to(q32))
    assert sim.size_classes() == [3]
    sim.load_state(to(scn.F0))
    out = [x.cpu().numpy() for x in sim.step(k, to(drops))]
    st = sim.state().cpu().numpy()
    sim.close()
    ro = discrete.Rollout(scn.H, scn.W, scn.F0, q32, scn.params.p_continue, seed=6)
    ob, od, odone = ro.step(k, np.ascontiguousarray(drops))
    np.testing.assert_array_equal(st, ro.F)
    np.testing.assert_array_equal(out[0], ob)
    np.testing.assert_array_equal(out[1], od)
    np.testing.assert_array_equal(out[2], odone)
