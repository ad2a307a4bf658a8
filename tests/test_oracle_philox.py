"""Pins for the oracle's Philox4x32-10 and its 24-bit uniforms.

Pin: Triton's independent Philox4x32-10 (triton.language.random.philox_impl,
run on the CPU by Triton's interpreter) must give the same words, bit for bit,
for random counters and keys, including the all-zero and all-ones extremes.
Statistics: the uniforms pass chi-square and Kolmogorov-Smirnov checks.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

from oracle import discrete

HERE = os.path.dirname(os.path.abspath(__file__))


def _triton_philox(ctr, key, tmp_path):
    pytest.importorskip("triton")
    i = tmp_path / "ctr.npy"
    o = tmp_path / "out.npy"
    np.save(i, ctr)
    env = dict(os.environ, TRITON_INTERPRET="1")
    subprocess.check_call([sys.executable, os.path.join(HERE, "_triton_philox.py"), str(i), str(o),
                           str(int(key[0])), str(int(key[1]))], env=env, timeout=600)
    return np.load(o)


@pytest.mark.parametrize("key", [(0, 0), (0xFFFFFFFF, 0xFFFFFFFF), (0x243F6A88, 0x85A308D3), (1234567, 0)])
def test_philox_matches_triton(key, tmp_path):
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2**32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    # structured counters as the model uses them: (cell, t, env, 4*episode+slot)
    ctr[2:10] = np.array([[c, 3, 5, 2] for c in range(8)], np.uint32)
    ours = discrete.philox(ctr, key)
    ref = _triton_philox(ctr, key, tmp_path)
    assert ours.dtype == np.uint32 and ref.dtype == np.uint32
    np.testing.assert_array_equal(ours, ref)


def test_uniform24_exact_grid():
    for w in [0, 1, 255, 256, 0xFFFFFFFF, 0x80000000, 12345678]:
        u = discrete.uniform24(w)
        assert 0.0 <= u < 1.0
        assert u * 2**24 == float(w >> 8)


def test_uniforms_statistics():
    n = 1 << 20
    ctr = np.zeros((n // 4, 4), np.uint32)
    ctr[:, 0] = np.arange(n // 4, dtype=np.uint32)
    ctr[:, 1] = 17
    ctr[:, 3] = 4 * 3 + 1
    w = discrete.philox(ctr, (42, 0)).reshape(-1)
    u = (w >> 8).astype(np.float64) * 2.0**-24
    counts, _ = np.histogram(u, bins=64, range=(0, 1))
    chi2 = ((counts - n / 64) ** 2 / (n / 64)).sum()
    assert stats.chi2.sf(chi2, 63) > 1e-4
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    # successive counters decorrelated
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 5.0 / np.sqrt(n)
