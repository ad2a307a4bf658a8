"""Pins for the two oracle functions the calibration and straight-through
tests rely on (CPU only).

calibration_loss (Section 4: cross-entropy on the spread shape plus the
squared error of 2-D average-pooled maps):
  * hand-worked values on maps whose pooled blocks and cross-entropy terms are
    known in closed form, in both orientations (a transposed pooling fails);
  * PyTorch's documented clamp of the log at -100 (a cell the prediction
    never reaches but the target does costs exactly 100);
  * the product's own loss equals it on random inputs, and its per-shard
    shares add up to the whole batch's value.

straight_through_grad (relaxed adjoint, Eqs. 5-10, chained backward along a
sampled trajectory, each step linearised at the state before it):
  * a two-step trajectory on a 1 x 2 grid worked by hand (a reversed chaining
    order or a linearisation at the state after a step changes the result);
  * with rates either 0 or so large that q rounds to 1 and p_continue in
    {0, 1}, the sampled trajectory of the C oracle is deterministic and equals
    the relaxed rollout state for state, so the straight-through gradient must
    equal autograd of the relaxed rollout (itself pinned to central
    differences).
"""
import math

import numpy as np
import pytest
import torch

from oracle import discrete, relaxed

f64 = torch.float64


# ---------------------------------------------------------------------------
# calibration_loss
# ---------------------------------------------------------------------------
def _two_block_case():
    """4 x 8 map, pool 4: left block pred 0.5 / target 1; right block pred
    0.25 / target 1 on its top two rows and 0 below."""
    pred = np.zeros((1, 4, 8))
    pred[..., :4] = 0.5
    pred[..., 4:] = 0.25
    tgt = np.zeros((1, 4, 8))
    tgt[..., :4] = 1.0
    tgt[:, :2, 4:] = 1.0
    # cross-entropy: 16 cells of -ln 0.5, 8 of -ln 0.25, 8 of -ln 0.75
    bce = (16 * math.log(2) + 8 * 2 * math.log(2) - 8 * math.log(0.75)) / 32
    # pooled: (0.5 - 1)^2 and (0.25 - 0.5)^2
    mse = (0.25 + 0.0625) / 2
    return pred, tgt, bce, mse


@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("w", [1.0, 2.5])
def test_calibration_loss_hand_worked(transpose, w):
    pred, tgt, bce, mse = _two_block_case()
    if transpose:
        pred, tgt = pred.transpose(0, 2, 1).copy(), tgt.transpose(0, 2, 1).copy()
    L = relaxed.calibration_loss(torch.as_tensor(1.0 - pred), torch.as_tensor(tgt), pool=4, w_mse=w)
    assert float(L) == pytest.approx(bce + w * mse, rel=1e-14)


def test_calibration_loss_batch_is_a_mean():
    pred, tgt, bce, mse = _two_block_case()
    # a second grid predicted exactly: cross-entropy of 0/1 predictions is 0
    pred2 = np.concatenate([pred, tgt], 0)
    tgt2 = np.concatenate([tgt, tgt], 0)
    L = relaxed.calibration_loss(torch.as_tensor(1.0 - pred2), torch.as_tensor(tgt2), pool=4)
    assert float(L) == pytest.approx((bce + mse) / 2, rel=1e-14)


def test_calibration_loss_log_clamp():
    p_un = torch.ones(1, 4, 4, dtype=f64)            # the fire reaches nothing
    tgt = torch.zeros(1, 4, 4, dtype=f64)
    tgt[0, 1, 2] = 1.0                               # ... but the target burned one cell
    L = relaxed.calibration_loss(p_un, tgt, pool=4)
    assert float(L) == pytest.approx(100.0 / 16 + (1.0 / 16) ** 2, rel=1e-14)


def test_product_loss_equals_oracle_and_shards_add_up():
    from paper_2512_06102_gb300 import relaxed as product
    rng = np.random.default_rng(3)
    N, H, W = 5, 12, 8
    pu = torch.as_tensor(rng.uniform(0.01, 0.99, size=(N, H, W)))
    tgt = torch.as_tensor(rng.uniform(0.0, 1.0, size=(N, H, W)))
    want = float(relaxed.calibration_loss(pu, tgt, pool=4))
    got = float(product.calibration_loss(pu.reshape(-1), tgt.reshape(-1), H, W, pool=4))
    assert got == pytest.approx(want, rel=1e-13)
    for cut in (0, 1, 3, 5):
        parts = [product.calibration_loss(pu[a:b].reshape(-1), tgt[a:b].reshape(-1), H, W, pool=4, n_total=N)
                 for a, b in ((0, cut), (cut, N))]
        assert float(sum(parts)) == pytest.approx(want, rel=1e-13)


# ---------------------------------------------------------------------------
# straight_through_grad
# ---------------------------------------------------------------------------
def _r_1x2(th, cA, cB):
    """Rates of a 1 x 2 grid (cells A, B): every direction into A is th0*cA,
    into B th0*cB (only the in-grid source counts: A -> B is direction 0, east;
    B -> A is direction 4, west)."""
    r = torch.zeros(1, 1, 2, 8, dtype=f64)
    r = r + torch.stack([th[0] * cA, th[0] * cB]).reshape(1, 1, 2, 1)
    return r


def test_straight_through_two_steps_by_hand():
    # x0 = [burning, can burn]; sampled x1 = [burned, burning]
    states = [np.array([[[2, 1]]], np.uint8), np.array([[[3, 2]]], np.uint8)]
    cA, cB, th0, pc = 0.7, 1.3, 0.9, 0.3
    theta = torch.tensor([th0, 0, 0, 0, 0, pc], dtype=f64)
    uA, uB, bA, bB = 0.4, -1.1, 1.0, -2.0
    a_un = torch.tensor([[[uA, uB]]], dtype=f64)
    a_b = torch.tensor([[[bA, bB]]], dtype=f64)
    g = relaxed.straight_through_grad(states, lambda th: _r_1x2(th, cA, cB), theta, a_un, a_b)
    # step 2 at x1 (nothing can ignite): the adjoint of p_burn is p_c times its
    # own, dL/dp_c collects bB; step 1 at x0: A spreads to B with rate th0*cB
    want_pc = bB + pc * bA
    want_th0 = cB * (pc * bB - uB) * math.exp(-th0 * cB)
    assert float(g[5]) == pytest.approx(want_pc, rel=1e-14)
    assert float(g[0]) == pytest.approx(want_th0, rel=1e-13)
    assert torch.all(g[1:5] == 0)


@pytest.mark.parametrize("pc", [0.0, 1.0])
def test_straight_through_equals_relaxed_when_deterministic(pc):
    rng = np.random.default_rng(7 + int(pc))
    H, W, T = 6, 7, 5
    F0 = rng.choice(np.array([0, 1, 1, 1, 3], np.uint8), size=(H, W))
    F0[2, 3] = 2
    F0[4, 1] = 2
    # per (target, direction): rate 0 or 60 (q = 1 - e^-60 is 1 in FP32 and
    # FP64, so ignition is certain and the relaxed step stays at 0/1);
    # no-fuel targets have rate 0 (their susceptibility is 0)
    big = (rng.random((H, W, 8)) < 0.6) * 60.0
    big[F0 == 0] = 0.0
    R = torch.as_tensor(big[None] / 0.58)
    r_of = lambda th: th[0] * R
    theta = torch.tensor([0.58, 0, 0, 0, 0, pc], dtype=f64)
    q = np.asarray(-np.expm1(-big), np.float32)
    assert set(np.unique(q)) <= {0.0, 1.0}
    # the sampled trajectory (C oracle), state before each step
    ro = discrete.Rollout([H], [W], F0.reshape(-1), q.reshape(-1, 8), pc, seed=5)
    states = []
    for _ in range(T):
        states.append(ro.F.reshape(1, H, W).copy())
        ro.step(1)
    # the relaxed rollout from the same start reproduces it state for state
    pu = torch.as_tensor((F0 <= 1).astype(np.float64))[None]
    pb = torch.as_tensor((F0 == 2).astype(np.float64))[None]
    th = theta.clone().requires_grad_(True)
    u, b = pu, pb
    for t in range(T):
        np.testing.assert_array_equal(u.detach().numpy(), (states[t] <= 1).astype(np.float64))
        np.testing.assert_array_equal(b.detach().numpy(), (states[t] == 2).astype(np.float64))
        u, b = relaxed.relaxed_step(u, b, r_of(th), th[5])
    Fend = ro.F.reshape(1, H, W)
    np.testing.assert_array_equal(u.detach().numpy(), (Fend <= 1).astype(np.float64))
    np.testing.assert_array_equal(b.detach().numpy(), (Fend == 2).astype(np.float64))
    a_un = torch.as_tensor(rng.standard_normal((1, H, W)))
    a_b = torch.as_tensor(rng.standard_normal((1, H, W)))
    L = (a_un * u).sum() + (a_b * b).sum()
    (want,) = torch.autograd.grad(L, [th])
    got = relaxed.straight_through_grad(states, r_of, theta, a_un, a_b)
    np.testing.assert_allclose(got.numpy(), want.numpy(), rtol=1e-12, atol=0)
    assert want[5] != 0 and (Fend >= 2).sum() > (F0 >= 2).sum() + 5      # the fire spread
