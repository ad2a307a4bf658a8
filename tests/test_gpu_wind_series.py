"""Wind as a time series on the GPU (Section 3: wind speed and direction are
indexed by the step).

The fused kernels evaluate the rates of Eqs. 1-4 per compared pair with the
wind row of the env's episode step.  Reference: the table path stepping one
step at a time with the probability table rebuilt from that step's wind (the
table kernel and the fused rate code compute bit-identical probabilities,
which the discrete-step tests pin).  States, counts and done flags must be
identical, for the resident and the tiled fused kernels, with drops, and with
auto-reset (the series restarts with every episode).  The oracle closes the
loop: with per-step tables from the FP64 oracle, the table path equals the C
oracle stepping with the same tables.
"""
import numpy as np
import pytest
import torch

from oracle import discrete, prob
from paper_2512_06102_gb300 import jwf, scenarios
from tests.gpu_util import make_sim, require_gpu, to

pytestmark = pytest.mark.gpu


def _series(T, N, seed):
    rng = np.random.default_rng(seed)
    ws = rng.uniform(0.0, 10.0, size=(T, N)).astype(np.float32)
    wd = rng.uniform(0.0, 2 * np.pi, size=(T, N)).astype(np.float32)
    return ws, wd


def _reference(scn, T, ws, wd, drops, seed, **kw):
    """Table path, one step per call, table rebuilt per step from each env's
    own episode step."""
    sim = make_sim(scn, seed=seed, **kw)
    sim.set_kernel(jwf.KERNEL_PLAIN)
    cls, dem = to(scn.cls), to(scn.dem)
    sim.load_state(to(scn.F0))
    outs = []
    N = scn.N
    for t in range(T):
        tt = sim.state_views()[1].cpu().numpy()
        row = np.minimum(tt, ws.shape[0] - 1)
        sim.precompute_probs(cls, dem, to(ws[row, np.arange(N)]), to(wd[row, np.arange(N)]))
        outs.append(sim.step(1, None if drops is None else to(drops[t:t + 1])))
    torch.cuda.synchronize()
    st = sim.state().cpu().numpy()
    res = [torch.cat([o[i] for o in outs]).cpu().numpy() for i in range(3)]
    sim.close()
    return st, res


def _fused(scn, T, ws, wd, drops, seed, kernel, **kw):
    sim = make_sim(scn, seed=seed, **kw)
    sim.set_terrain(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    sim.set_wind_series(to(ws), to(wd))
    sim.set_kernel(kernel)
    sim.load_state(to(scn.F0))
    out = sim.step(T, None if drops is None else to(drops))
    torch.cuda.synchronize()
    st = sim.state().cpu().numpy()
    res = [x.cpu().numpy() for x in out]
    sim.close()
    return st, res


@pytest.mark.parametrize("kernel,shape,N", [(jwf.KERNEL_FUSED, (40, 56), 6),
                                            (jwf.KERNEL_TILED_FUSED, (150, 300), 2)])
def test_series_equals_per_step_tables(kernel, shape, N):
    require_gpu()
    H, W = shape
    T = 24
    scn = scenarios.make_scenario(H, W, N=N, seed=31)
    ws, wd = _series(T, N, 5)
    drops = scenarios.drops(T, scn.H, scn.W, seed=3)
    a = _fused(scn, T, ws, wd, drops, 7, kernel)
    b = _reference(scn, T, ws, wd, drops, 7)
    np.testing.assert_array_equal(a[0], b[0])
    for x, y in zip(a[1], b[1]):
        np.testing.assert_array_equal(x, y)
    assert int(a[1][1][-1].sum()) > 0


def test_series_restarts_with_the_episode():
    require_gpu()
    H, W, N, T = 32, 32, 8, 40
    scn = scenarios.make_scenario(H, W, N=N, seed=32)
    ws, wd = _series(9, N, 6)       # shorter than the run: the last row holds
    a = _fused(scn, T, ws, wd, None, 3, jwf.KERNEL_FUSED, auto_reset=True, t_max=7)
    b = _reference(scn, T, ws, wd, None, 3, auto_reset=True, t_max=7)
    np.testing.assert_array_equal(a[0], b[0])
    for x, y in zip(a[1], b[1]):
        np.testing.assert_array_equal(x, y)
    assert a[1][2].sum() >= N * (T // 7)      # every env restarted several times


def test_series_needs_a_fused_kernel():
    require_gpu()
    scn = scenarios.make_scenario(24, 24, N=2, seed=33)
    ws, wd = _series(4, 2, 7)
    sim = make_sim(scn)
    sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    sim.set_wind_series(to(ws), to(wd))
    sim.set_kernel(jwf.KERNEL_RESIDENT)
    sim.load_state(to(scn.F0))
    with pytest.raises(jwf.JwfError):
        sim.step(2)
    sim.set_wind_series(None)
    sim.step(2)
    sim.close()


def test_table_path_with_oracle_tables_per_step():
    require_gpu()
    H, W, N, T = 30, 34, 3, 12
    scn = scenarios.make_scenario(H, W, N=N, seed=34)
    ws, wd = _series(T, N, 8)
    p = scn.params.as_dict()
    sim = make_sim(scn, seed=9)
    sim.set_kernel(jwf.KERNEL_PLAIN)
    sim.load_state(to(scn.F0))
    ro = None
    for t in range(T):
        q = np.concatenate([prob.table_f32(scn.env(e, scn.cls)[None], scn.env(e, scn.dem)[None], ws[t, e:e + 1],
                                           wd[t, e:e + 1], p, scn.params.cell_size)[0].reshape(-1, 8)
                            for e in range(N)])
        sim.set_probs(to(q))
        gb, gd, gdone = [x.cpu().numpy() for x in sim.step(1)]
        if ro is None:
            ro = discrete.Rollout(scn.H, scn.W, scn.F0, q, scn.params.p_continue, seed=9)
        ro.q = np.ascontiguousarray(q, np.float32)
        ob, od, odone = ro.step(1)
        np.testing.assert_array_equal(gb, ob)
        np.testing.assert_array_equal(gd, od)
        np.testing.assert_array_equal(gdone, odone)
    np.testing.assert_array_equal(sim.state().cpu().numpy(), ro.F)
    sim.close()
