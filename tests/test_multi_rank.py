"""Multi-rank host logic on CPU (gloo, world size 2).

  * grids shard into contiguous ranges that cover the batch once and are
    balanced by cell count;
  * the calibration gradient (Section 4) sharded over two ranks and summed
    with an all-reduce equals the gradient of the whole batch (the loss is a
    sum over grids), computed with the FP64 oracle;
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


def _oracle_grad(scn, envs, T):
    from oracle import prob
    from oracle import relaxed as orl
    C = len(scn.params.mu_veg)
    p = scn.params
    th = torch.tensor([p.p_base, p.alpha_w1, p.alpha_w2, p.alpha_s, p.alpha_gamma, p.p_continue]
                      + list(p.mu_veg) + list(p.mu_den), dtype=f64, requires_grad=True)
    if len(envs) == 0:
        return torch.zeros(6 + 2 * C, dtype=f64)
    cls = torch.as_tensor(np.stack([scn.env(e, scn.cls) for e in envs])).long()
    dem = torch.as_tensor(np.stack([scn.env(e, scn.dem) for e in envs]).astype(np.float64))
    r = prob.rates(cls, dem, torch.as_tensor(scn.wind_speed[envs].astype(np.float64)),
                   torch.as_tensor(scn.wind_dir[envs].astype(np.float64)), th[0], th[1], th[2], th[3], th[4],
                   th[6:6 + C], th[6 + C:6 + 2 * C], p.cell_size)
    F0 = torch.as_tensor(np.stack([scn.env(e, scn.F0) for e in envs]).astype(np.int64))
    pb = (F0 == 2).to(f64)
    pu = 1.0 - pb
    ou, ob = orl.relaxed_rollout(pu, pb, r, th[5], T)
    loss = (1.0 - ou).sum() + 0.5 * ob.sum()
    (g,) = torch.autograd.grad(loss, [th])
    return g


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        scn = scenarios.make_scenario(12, 11, N=5, seed=4)
        cells = scn.H.astype(np.int64) * scn.W
        a, b = shard.shard_ranges(cells, world)[rank]
        g = _oracle_grad(scn, list(range(a, b)), T=6)
        shard.allreduce_sum_(g)
        # max over ranks, as the benchmark reduces its timings
        t = torch.tensor([float(rank + 1)], dtype=f64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            full = _oracle_grad(scn, list(range(scn.N)), T=6)
            out.put((g.numpy(), full.numpy(), float(t.item())))
    finally:
        dist.destroy_process_group()


def test_sharded_calibration_gradient_equals_whole_batch():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    g, full, tmax = q.get()
    np.testing.assert_allclose(g, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())
    assert tmax == 2.0
    assert np.abs(full).max() > 0
