"""Multi-rank host logic on CPU (gloo, world size 2).

  * grids shard into contiguous ranges that cover the batch once and are
    balanced by cell count;
  * the calibration step of the product (calibrate.sharded_loss_grad on each
    rank's share of relaxed.calibration_loss, one all-reduce) gives the whole
    batch's loss and gradient, with deliberately unequal shards and with an
    empty one; the relaxed rollout under it is the FP64 oracle's;
  * the benchmark's max-over-ranks timing reduces across processes.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2512_06102_gb300 import scenarios, shard

f64 = torch.float64


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_ranges_cover_and_balance():
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 8):
        for n in (0, 1, 5, 37, 1000):
            cells = rng.integers(32 * 32, 512 * 512, size=n)
            rs = shard.shard_ranges(cells, world)
            assert len(rs) == world
            assert rs[0][0] == 0 and rs[-1][1] == n
            for (a, b), (c, d) in zip(rs[:-1], rs[1:]):
                assert b == c and a <= b
            if n >= 8 * world:
                loads = [int(cells[a:b].sum()) for a, b in rs]
                # each rank within one grid of the even split
                assert max(loads) - min(loads) <= 2 * int(cells.max())


SHARDS = {"unequal": [(0, 1), (1, 5)], "empty": [(0, 0), (0, 5)], "balanced": None}


def _local_loss(scn, envs, target, z, theta0, scale, T, n_total):
    """This rank's share of the Section 4 loss of the FP64 oracle rollout,
    as a function of z (theta = theta0 + scale * z, as calibrate.fit)."""
    from oracle import prob
    from oracle import relaxed as orl
    from paper_2512_06102_gb300 import relaxed as product
    if len(envs) == 0:
        return None
    C = len(scn.params.mu_veg)
    th = theta0 + scale * z
    cls = torch.as_tensor(np.stack([scn.env(e, scn.cls) for e in envs])).long()
    dem = torch.as_tensor(np.stack([scn.env(e, scn.dem) for e in envs]).astype(np.float64))
    r = prob.rates(cls, dem, torch.as_tensor(scn.wind_speed[envs].astype(np.float64)),
                   torch.as_tensor(scn.wind_dir[envs].astype(np.float64)), th[0], th[1], th[2], th[3], th[4],
                   th[6:6 + C], th[6 + C:6 + 2 * C], scn.params.cell_size)
    F0 = torch.as_tensor(np.stack([scn.env(e, scn.F0) for e in envs]).astype(np.int64))
    pb = (F0 == 2).to(f64)
    ou, _ = orl.relaxed_rollout(1.0 - pb, pb, r, th[5], T)
    H, W = int(scn.H[0]), int(scn.W[0])
    return product.calibration_loss(ou.reshape(-1), target[envs].reshape(-1), H, W, pool=4, n_total=n_total)


def _problem():
    from paper_2512_06102_gb300 import calibrate
    scn = scenarios.make_scenario(12, 8, N=5, seed=4)
    C = len(scn.params.mu_veg)
    theta0 = calibrate.theta_of(scn.params, C)
    scale = theta0.abs().clamp_min(0.05)
    target = torch.as_tensor(np.random.default_rng(9).uniform(0.0, 1.0, size=(5, 12, 8)))
    free = torch.ones_like(theta0)          # every parameter, p_continue included
    return scn, theta0, scale, target, free


def _sharded(rank, world, ranges):
    from paper_2512_06102_gb300 import calibrate
    scn, theta0, scale, target, free = _problem()
    if ranges is None:
        cells = scn.H.astype(np.int64) * scn.W
        ranges = shard.shard_ranges(cells, world)
    a, b = ranges[rank]
    n_total = shard.global_count(b - a)
    z = torch.zeros_like(theta0, requires_grad=True)
    loss = _local_loss(scn, list(range(a, b)), target, z, theta0, scale, T=6, n_total=n_total)
    lv = calibrate.sharded_loss_grad(z, loss, free)
    return n_total, lv, z.grad.detach().clone()


def _whole():
    from paper_2512_06102_gb300 import calibrate
    scn, theta0, scale, target, free = _problem()
    z = torch.zeros_like(theta0, requires_grad=True)
    loss = _local_loss(scn, list(range(scn.N)), target, z, theta0, scale, T=6, n_total=None)
    lv = calibrate.sharded_loss_grad(z, loss, free)          # one process: no reduction
    return lv, z.grad.detach().clone()


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {k: _sharded(rank, world, v) for k, v in SHARDS.items()}
        # max over ranks, as the benchmark reduces its timings
        t = torch.tensor([float(rank + 1)], dtype=f64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            out.put(({k: (n, lv, g.numpy()) for k, (n, lv, g) in res.items()}, float(t.item())))
    finally:
        dist.destroy_process_group()


def test_sharded_calibration_step_equals_whole_batch():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res, tmax = q.get()
    lv_full, g_full = _whole()
    g_full = g_full.numpy()
    assert np.abs(g_full).max() > 0
    for name, (n_total, lv, g) in res.items():
        assert n_total == 5, name
        assert lv == pytest.approx(lv_full, rel=1e-12), name
        np.testing.assert_allclose(g, g_full, rtol=1e-12, atol=1e-12 * np.abs(g_full).max(), err_msg=name)
    assert tmax == 2.0


def test_sharded_step_without_process_group_is_the_whole_batch():
    """One process: global_count is the local count and the reduction is the
    identity, so the step is the plain whole-batch step."""
    assert shard.global_count(7) == 7
    g = torch.tensor([1.0, -2.0], dtype=f64)
    assert shard.reduce_loss_and_grad_(g, torch.tensor(3.5, dtype=f64)) == 3.5
    assert g.tolist() == [1.0, -2.0]


def test_fit_on_an_empty_shard_takes_part_without_a_simulator():
    """A rank whose shard holds no grids calls calibrate.fit without a
    simulator: it contributes a zero loss and gradient, and (with no other
    rank) its parameters stay where they started."""
    from paper_2512_06102_gb300 import calibrate
    theta0 = calibrate.theta_of(scenarios.Params(), scenarios.N_CLASSES)
    theta, losses = calibrate.fit(None, None, None, None, theta0, T=3, iters=2)
    assert losses == [0.0, 0.0]
    assert torch.equal(theta, theta0)
