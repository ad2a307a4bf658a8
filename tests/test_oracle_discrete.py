"""Pins for the discrete-step oracle (Section 3 "Stochastic update", Section 4 action).

  * Chebyshev square: with every probability 1, one centre fire and any
    p_continue, the burning-or-burned set after t steps is exactly the square
    of Chebyshev radius t (clipped to the grid);
  * zero spread: with every probability 0 the burning set only shrinks;
  * no-fuel cells never ignite, burned cells never change;
  * p_continue = 1 keeps every fire burning, p_continue = 0 burns every fire out;
  * the tanker mask turns only burning cells into burned ones, before the
    spread (a doused cell ignites nobody in that step);
  * Eq. 4 by Monte Carlo: over 10^6 independent trials on a 5x5 grid, the
    ignition frequency of each target is within 4 sigma of
    1 - exp(-sum of incoming rates), and the remain-burning frequency within
    4 sigma of p_continue;
  * exact law by brute force: on a 3x3 grid every joint outcome of the active
    draws is enumerated; the oracle's outcome frequencies over 10^6 trials
    match the exact probabilities within 4 sigma.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import discrete, prob

DX, DR = prob.DX, prob.DR


def _cheb(H, W, cy, cx, t):
    y, x = np.mgrid[0:H, 0:W]
    return np.maximum(abs(y - cy), abs(x - cx)) <= t


@pytest.mark.parametrize("p_c", [0.0, 0.5, 1.0])
@pytest.mark.parametrize("shape,centre", [((33, 33), (16, 16)), ((20, 37), (3, 30))])
def test_chebyshev_square(p_c, shape, centre):
    H, W = shape
    F = np.ones((H, W), np.uint8)
    F[centre] = 2
    q = np.ones((H, W, 8), np.float32)
    for t in range(1, 25):
        F, nb, nd = discrete.step(F, q, p_c, seed=11, t=t - 1)
        lit = (F == 2) | (F == 3)
        np.testing.assert_array_equal(lit, _cheb(H, W, centre[0], centre[1], t))
        assert nb == int((F == 2).sum()) and nd == int((F == 3).sum())
        if p_c == 1.0:
            assert (F != 3).all()
        if p_c == 0.0:
            # only the newest ring burns
            np.testing.assert_array_equal(F == 2, lit & ~_cheb(H, W, centre[0], centre[1], t - 1))


def test_zero_probability_no_spread():
    rng = np.random.default_rng(1)
    F = rng.integers(0, 4, size=(30, 30)).astype(np.uint8)
    q = np.zeros((30, 30, 8), np.float32)
    for t in range(20):
        G, _, _ = discrete.step(F, q, 0.7, seed=2, t=t)
        assert not ((F != 2) & (G == 2)).any()
        F = G


def test_nofuel_never_ignites_burnt_absorbing():
    rng = np.random.default_rng(5)
    for trial in range(20):
        F = rng.integers(0, 4, size=(24, 24)).astype(np.uint8)
        q = rng.random((24, 24, 8)).astype(np.float32)
        q[rng.random((24, 24, 8)) < 0.3] = 1.0
        G, _, _ = discrete.step(F, q, float(rng.random()), seed=trial, t=trial)
        assert (G[F == 0] == 0).all()
        assert (G[F == 3] == 3).all()
        assert set(np.unique(G[F == 1])) <= {1, 2}
        assert set(np.unique(G[F == 2])) <= {2, 3}


def test_action_before_spread():
    H = W = 9
    F = np.ones((H, W), np.uint8)
    F[4, 4] = 2
    q = np.ones((H, W, 8), np.float32)
    mask = discrete.drop_mask(H, W, 4, 4, 1)
    G, nb, nd = discrete.step(F, q, 1.0, mask=mask)
    assert G[4, 4] == 3 and nb == 0 and nd == 1          # doused before it could spread
    assert (G[mask.astype(bool) & (F == 1)] == 1).all()  # water does not touch unburned fuel
    m = discrete.drop_mask(H, W, 0, 8, 1)                # clipped at a corner
    assert m.sum() == 4 and m[7:, :2].all()
    assert discrete.drop_mask(H, W, -1, -1, 1).sum() == 0


def test_eq4_monte_carlo_5x5():
    rng = np.random.default_rng(9)
    H = W = 5
    F = np.ones((H, W), np.uint8)
    F[1, 1] = F[1, 3] = F[3, 2] = F[2, 0] = 2
    F[0, 4] = 0
    r = rng.uniform(0.05, 1.2, size=(H, W, 8))
    q = (-np.expm1(-r)).astype(np.float32)
    n = 1_000_000
    p_c = 0.37
    out = discrete.mc_outcomes(F, q, p_c, n, seed=123)
    for y in range(H):
        for x in range(W):
            freq_burn = (out[:, y, x] == 2).mean()
            if F[y, x] == 1:
                lam = sum(r[y, x, d] for d in range(8)
                          if 0 <= y - DR[d] < H and 0 <= x - DX[d] < W and F[y - DR[d], x - DX[d]] == 2)
                p = -math.expm1(-lam)                   # Eq. 4
            elif F[y, x] == 2:
                p = p_c
            else:
                p = 0.0
            sigma = math.sqrt(max(p * (1 - p), 1e-12) / n)
            assert abs(freq_burn - p) <= 4 * sigma + 1e-6, (y, x, freq_burn, p)


def _brute_force_law(F, q, p_c):
    """Exact distribution of the post-step grid by enumerating every active draw."""
    H, W = F.shape
    draws = []   # (kind, cell, prob)
    for y in range(H):
        for x in range(W):
            if F[y, x] == 1:
                for d in range(8):
                    uy, ux = y - DR[d], x - DX[d]
                    if 0 <= uy < H and 0 <= ux < W and F[uy, ux] == 2:
                        draws.append(("ign", (y, x), float(q[y, x, d])))
            elif F[y, x] == 2:
                draws.append(("cont", (y, x), p_c))
    law = {}
    for bits in itertools.product((0, 1), repeat=len(draws)):
        pr = 1.0
        G = F.copy()
        G[F == 2] = 3
        for b, (kind, cell, p) in zip(bits, draws):
            pr *= p if b else (1 - p)
            if b:
                G[cell] = 2
        key = G.tobytes()
        law[key] = law.get(key, 0.0) + pr
    return law


def test_brute_force_law_3x3():
    F = np.array([[2, 1, 1], [1, 2, 0], [3, 1, 1]], np.uint8)
    rng = np.random.default_rng(4)
    q = rng.uniform(0.1, 0.9, size=(3, 3, 8)).astype(np.float32)
    p_c = 0.6
    law = _brute_force_law(F, q, p_c)
    assert abs(sum(law.values()) - 1.0) < 1e-12
    n = 1_000_000
    out = discrete.mc_outcomes(F, q, p_c, n, seed=77, t=5, episode=2)
    keys, counts = np.unique(out.reshape(n, -1), axis=0, return_counts=True)
    seen = {k.tobytes(): c / n for k, c in zip(keys, counts)}
    assert set(seen) <= set(law), "oracle produced an outcome of probability zero"
    for k, p in law.items():
        f = seen.get(k, 0.0)
        sigma = math.sqrt(p * (1 - p) / n)
        assert abs(f - p) <= 4 * sigma + 1e-6


def test_rollout_auto_reset_and_counts():
    H = W = 8
    F0 = np.ones((2, H, W), np.uint8)
    F0[:, 4, 4] = 2
    q = np.zeros((2, H, W, 8), np.float32)            # nothing spreads
    ro = discrete.Rollout([H, H], [W, W], F0.reshape(-1), q.reshape(-1, 8), p_continue=0.0,
                          seed=0, t_max=0, auto_reset=True)
    b, d, done = ro.step(3)
    # p_continue = 0: the fire burns out in the first step -> done -> reset
    assert (b[0] == 0).all() and (d[0] == 1).all() and (done[0] == 1).all()
    assert (ro.episode == 3).all() and (ro.t == 0).all()
    np.testing.assert_array_equal(ro.F, F0.reshape(-1))
    ro2 = discrete.Rollout([H, H], [W, W], F0.reshape(-1), q.reshape(-1, 8), p_continue=1.0,
                           seed=0, t_max=2, auto_reset=False)
    b, d, done = ro2.step(3)
    assert done[:, 0].tolist() == [0, 1, 1] and (ro2.t == 3).all()


def test_packed_format_hand_worked():
    # states 1, 2, 3, 0 | 3 -> byte 0 = 1 + 2*4 + 3*16 + 0*64 = 57, byte 1 = 3
    P = discrete.pack_states(np.array([1, 2, 3, 0, 3], np.uint8))
    assert P.tolist() == [57, 3]
    assert discrete.pack_states(np.zeros(0, np.uint8)).size == 0
    assert discrete.pack_states(np.full(8, 3, np.uint8)).tolist() == [255, 255]


def test_packed_format_roundtrip():
    rng = np.random.default_rng(0)
    for n in (1, 2, 3, 4, 5, 31, 33, 1000):
        F = rng.integers(0, 4, size=n).astype(np.uint8)
        P = discrete.pack_states(F)
        assert P.size == (n + 3) // 4
        np.testing.assert_array_equal(discrete.unpack_states(P, n), F)
        # every cell's two bits, read one by one
        for i in range(n):
            assert (int(P[i // 4]) >> (2 * (i % 4))) & 3 == F[i]


def test_masked_rollout_equals_drop_rollout():
    """The rollout with each step's action as a cell mask (Section 4: water on
    a burning cell burns it out before the spread) reproduces the drop rollout
    bit for bit when the masks are the drops' 3x3 footprints, on a ragged
    batch with auto-reset; all-zero masks reproduce the rollout without
    action."""
    from paper_2512_06102_gb300 import scenarios
    rng = np.random.default_rng(17)
    sides_h, sides_w = [9, 14, 6], [12, 7, 10]
    scn = scenarios.make_scenario(sides_h, sides_w, seed=17)
    q = rng.uniform(0.0, 0.9, size=(scn.F0.size, 8)).astype(np.float32)
    k = 25
    drops = scenarios.drops(k, scn.H, scn.W, seed=17)
    masks = np.zeros((k, scn.F0.size), np.uint8)
    for t in range(k):
        for e in range(scn.N):
            m = discrete.drop_mask(int(scn.H[e]), int(scn.W[e]), int(drops[t, e, 0]), int(drops[t, e, 1]))
            masks[t, scn.offsets[e]:scn.offsets[e + 1]] = m.reshape(-1)
    kw = dict(p_continue=0.6, seed=3, t_max=9, auto_reset=True)
    a = discrete.Rollout(scn.H, scn.W, scn.F0, q, **kw)
    b = discrete.Rollout(scn.H, scn.W, scn.F0, q, **kw)
    oa = a.step(k, drops)
    ob = b.step_masks(masks)
    np.testing.assert_array_equal(a.F, b.F)
    for x, y in zip(oa, ob):
        np.testing.assert_array_equal(x, y)
    assert (a.episode >= 1).any()
    c = discrete.Rollout(scn.H, scn.W, scn.F0, q, **kw)
    d = discrete.Rollout(scn.H, scn.W, scn.F0, q, **kw)
    oc = c.step(k, None)
    od = d.step_masks(np.zeros_like(masks))
    np.testing.assert_array_equal(c.F, d.F)
    for x, y in zip(oc, od):
        np.testing.assert_array_equal(x, y)
