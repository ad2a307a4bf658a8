"""Helpers shared by the GPU parity tests (the tests call libjwf through its C ABI)."""
import numpy as np
import pytest
import torch


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_06102_gb300 import build
    build.build()       # a GPU machine without the library fails here, loudly


def dev():
    return torch.device("cuda", torch.cuda.current_device())


def to(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def oracle_tables(scn):
    """(q32, r32, q64, r64) as [cells, 8] from the FP64 oracle, env by env."""
    from oracle import prob
    qs32, rs32, qs64, rs64 = [], [], [], []
    p = scn.params.as_dict()
    for e in range(scn.N):
        a = prob.table_f32(scn.env(e, scn.cls)[None], scn.env(e, scn.dem)[None],
                           scn.wind_speed[e:e + 1], scn.wind_dir[e:e + 1], p, scn.params.cell_size)
        for lst, x in zip((qs32, rs32, qs64, rs64), a):
            lst.append(x.reshape(-1, 8))
    return tuple(np.concatenate(x) for x in (qs32, rs32, qs64, rs64))


def make_sim(scn, seed=0, **kw):
    from paper_2512_06102_gb300 import jwf, scenarios
    sim = jwf.Sim(scn.H, scn.W, n_classes=len(scn.params.mu_veg), seed=seed, **kw)
    sim.set_params(scn.params)
    return sim
