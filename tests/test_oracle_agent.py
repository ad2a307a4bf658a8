"""Pins of the agent-environment oracle (Section 4's air-tanker scenario).

The paper fixes the reward (a penalty per burning cell, +10 for an
extinguished fire) and that water turns burning cells into burned ones;
movement, valve, window and restart are this build's readings, checked here
against hand-worked cases."""
import numpy as np

from oracle import agent, discrete


def _env(F, q=0.0, p_c=1.0, **kw):
    H, W = F.shape
    qt = np.full((H * W, 8), q, np.float32)
    return agent.TankerOracle([H], [W], F.reshape(-1), qt, p_c, **kw)


def test_moves_clamp_and_stay():
    F = np.zeros((5, 6), np.uint8)
    F[0, 0] = 2                          # keeps the episode alive (p_continue = 1, nothing to ignite)
    env = _env(F, random_fire=False, water0=0)
    env.agent[0] = (2, 2, 0)
    path = []
    for a in [1, 1, 1, 2, 2, 2, 2, 3, 4, 0, 9, -3, 17]:
        env.step([a])
        path.append(tuple(env.agent[0, :2]))
    assert path == [(2, 1), (2, 0), (2, 0), (3, 0), (4, 0), (5, 0), (5, 0), (5, 1), (4, 1), (4, 1), (3, 1),
                    (3, 1), (3, 1)]


def test_valve_water_and_extinction_reward():
    F = np.ones((5, 5), np.uint8)
    F[2, 2] = 2
    env = _env(F, random_fire=False, water0=2, burn_penalty=0.5)
    env.agent[0] = (0, 0, 2)
    obs, r, d = env.step([2])            # move east, valve closed: the fire burns on
    assert tuple(env.agent[0]) == (1, 0, 2) and r[0] == np.float32(-0.5) and d[0] == 0
    obs, r, d = env.step([8])            # south + valve: drop at (1, 1) covers (2, 2)
    assert d[0] == 1 and r[0] == np.float32(10.0)
    # the episode restarted: fresh water, a position on the grid
    assert env.agent[0, 2] == 2
    assert 0 <= env.agent[0, 0] < 5 and 0 <= env.agent[0, 1] < 5


def test_no_water_no_drop():
    F = np.ones((5, 5), np.uint8)
    F[2, 2] = 2
    env = _env(F, random_fire=False, water0=0, burn_penalty=0.25)
    env.agent[0] = (2, 2, 0)
    _, r, d = env.step([5])              # valve open but the tank is empty
    assert d[0] == 0 and r[0] == np.float32(-0.25) and env.agent[0, 2] == 0


def test_observation_window_with_outside_marker():
    F = np.arange(35, dtype=np.uint8).reshape(5, 7) % 4
    env = _env(F, random_fire=False)
    env.agent[0] = (0, 1, 3)
    o = env.obs()[0]
    ref = np.full((5, 5), 255, np.uint8)
    for i in range(5):
        for j in range(5):
            y, x = 1 - 2 + i, 0 - 2 + j
            if 0 <= y < 5 and 0 <= x < 7:
                ref[i, j] = F[y, x]
    np.testing.assert_array_equal(o, ref)


def test_restart_draws_and_random_ignition():
    F = np.zeros((6, 9), np.uint8)
    F[4, 7] = 1                          # the only can-burn cell: the ignition must land there
    env = _env(F, random_fire=True, seed=12345, water0=7)
    env.reset()
    w = discrete.philox(np.array([[0, 0, 0, 3]], np.uint32), (12345, 0))[0]
    u = [np.float32(int(x) >> 8) * np.float32(2.0 ** -24) for x in w]
    assert tuple(env.agent[0]) == (int(u[0] * np.float32(9)), int(u[1] * np.float32(6)), 7)
    assert env.ro.env_state(0)[4, 7] == 2 and (env.ro.env_state(0) == 2).sum() == 1
    # positions are uniform over the grid across restarts
    xs = []
    for ep in range(400):
        env.ro.episode[0] = ep
        env._restart(0)
        xs.append(tuple(env.agent[0, :2]))
    xs = np.array(xs)
    assert xs[:, 0].min() == 0 and xs[:, 0].max() == 8 and xs[:, 1].min() == 0 and xs[:, 1].max() == 5
