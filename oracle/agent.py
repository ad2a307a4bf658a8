"""Oracle of the air-tanker agent environment (Section 4).

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product path.

Section 4 trains an air-tanker agent: it receives partial egocentric
observations, controls a valve that drops a limited amount of water, water
turns burning cells into burned cells, each step costs a penalty
proportional to the number of burning cells, putting the fire out completely
earns +10, and fire and agent positions are randomised at the start of an
episode.  The paper gives no more detail; the readings written out here (and
listed with the design notes) are:
  * action a in [0, 10): move = a % 5 (0 stay, 1 north = row - 1, 2 east =
    column + 1, 3 south, 4 west), clamped to the grid; valve open iff a >= 5;
    other values count as 0;
  * an open valve with water left drops water on the drop footprint centred on
    the agent's new cell (the step's action, applied before the spread) and
    uses one unit;
  * reward = -burn_penalty * (burning cells after the step) + 10 if none;
  * observation = the obs_k x obs_k states centred on the agent, 255 outside;
  * restart: Philox4x32-10 with the step's key and counter (0, 0, env,
    4 * episode + 3): x = floor(u(w0) W), y = floor(u(w1) H) (the products in
    float32), water = water0; with random_fire the first can-burn cell at or
    after cell floor(u(w2) H W), row-major and wrapping, starts burning.
The spread itself is the C oracle's discrete step (oracle.discrete.Rollout,
auto-reset on).
"""
from __future__ import annotations

import numpy as np

from . import discrete


def _u24(w) -> np.float32:
    return np.float32(int(w) >> 8) * np.float32(2.0 ** -24)


class TankerOracle:
    def __init__(self, H, W, F0, q, p_continue, seed: int = 0, t_max: int = 0, radius: int = 1, water0: int = 10,
                 obs_k: int = 5, burn_penalty: float = 0.01, random_fire: bool = True):
        self.ro = discrete.Rollout(H, W, F0, q, p_continue, seed=seed, t_max=t_max, auto_reset=True, radius=radius)
        self.N = self.ro.N
        self.seed = int(seed)
        self.water0 = int(water0)
        self.obs_k = int(obs_k)
        self.burn_penalty = np.float32(burn_penalty)
        self.random_fire = bool(random_fire)
        self.agent = np.zeros((self.N, 3), np.int32)

    def _key(self):
        return (self.seed & 0xFFFFFFFF, (self.seed >> 32) & 0xFFFFFFFF)

    def _restart(self, e: int):
        H, W = int(self.ro.H[e]), int(self.ro.W[e])
        ctr = np.array([[0, 0, e, 4 * int(self.ro.episode[e]) + 3]], np.uint32)
        w = discrete.philox(ctr, self._key())[0]
        self.agent[e] = (min(int(_u24(w[0]) * np.float32(W)), W - 1), min(int(_u24(w[1]) * np.float32(H)), H - 1),
                         self.water0)
        if self.random_fire:
            n = H * W
            start = min(int(_u24(w[2]) * np.float32(n)), n - 1)
            F = self.ro.F[self.ro.off[e]:self.ro.off[e] + n]
            for k in range(n):
                c = (start + k) % n
                if F[c] == 1:
                    F[c] = 2
                    break

    def obs(self) -> np.ndarray:
        k, r = self.obs_k, self.obs_k // 2
        out = np.full((self.N, k, k), 255, np.uint8)
        for e in range(self.N):
            H, W = int(self.ro.H[e]), int(self.ro.W[e])
            F = self.ro.env_state(e)
            x, y = int(self.agent[e, 0]), int(self.agent[e, 1])
            for i in range(k):
                for j in range(k):
                    yy, xx = y - r + i, x - r + j
                    if 0 <= yy < H and 0 <= xx < W:
                        out[e, i, j] = F[yy, xx]
        return out

    def reset(self) -> np.ndarray:
        for e in range(self.N):
            self._restart(e)
        return self.obs()

    def step(self, actions):
        """actions int [N] -> (obs, reward float32 [N], done uint8 [N])."""
        drops = np.full((1, self.N, 2), -1, np.int32)
        for e in range(self.N):
            a = int(actions[e])
            if a < 0 or a >= 10:
                a = 0
            H, W = int(self.ro.H[e]), int(self.ro.W[e])
            x, y, water = (int(v) for v in self.agent[e])
            move = a % 5
            y += -1 if move == 1 else (1 if move == 3 else 0)
            x += 1 if move == 2 else (-1 if move == 4 else 0)
            x = min(max(x, 0), W - 1)
            y = min(max(y, 0), H - 1)
            if a >= 5 and water > 0:
                drops[0, e] = (x, y)
                water -= 1
            self.agent[e] = (x, y, water)
        burning, _, done = self.ro.step(1, drops)
        nb = burning[0]
        reward = (-self.burn_penalty * nb.astype(np.float32) + np.where(nb == 0, np.float32(10.0), np.float32(0.0)))
        for e in range(self.N):
            if done[0, e]:
                self._restart(e)
        return self.obs(), reward.astype(np.float32), done[0].copy()
