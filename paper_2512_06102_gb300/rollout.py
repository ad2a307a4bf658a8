"""RL rollouts on libjwf captured as one CUDA graph.

A rollout of T steps issues jwf_step calls of `steps_per_launch` steps (1 for
an agent that acts every step; more when the actions are drawn in advance,
as for random tanker drops) and computes each step's reward from the per-env
counts (Section 4: a penalty proportional to the number of burning cells,
+10 when the fire is completely extinguished).  With JWF_AUTO_RESET the kernels restart done
envs themselves, so the whole rollout has no host synchronisation and is
captured once (torch.cuda.CUDAGraph) and replayed; the only host work per
rollout is one graph launch.
"""
from __future__ import annotations

import torch

from . import jwf


def reward(burning: torch.Tensor, prev_burning: torch.Tensor, burn_penalty: float = 0.01,
           extinguish_bonus: float = 10.0) -> torch.Tensor:
    """-c * (burning cells) + 10 if the step put out the last burning cell."""
    out = -burn_penalty * burning.to(torch.float32)
    return out + extinguish_bonus * ((burning == 0) & (prev_burning > 0)).to(torch.float32)


class GraphRollout:
    """T steps of `sim` with drops [T, N, 2] (int32, device), captured once.

    Capturing runs one warm-up step eagerly first (it advances the Sim by one
    step): load or reset the state before run()."""

    def __init__(self, sim: jwf.Sim, T: int, drops: torch.Tensor, capture: bool = True,
                 burn_penalty: float = 0.01, steps_per_launch: int = 1):
        self.sim, self.T = sim, int(T)
        self.k = max(1, min(int(steps_per_launch), self.T))
        dev = drops.device
        N = sim.N
        self.drops = drops.contiguous()
        self.burning = torch.zeros((T, N), dtype=torch.int32, device=dev)
        self.burnt = torch.zeros((T, N), dtype=torch.int32, device=dev)
        self.done = torch.zeros((T, N), dtype=torch.uint8, device=dev)
        self.rewards = torch.zeros((T, N), dtype=torch.float32, device=dev)
        self.prev = torch.zeros(N, dtype=torch.int32, device=dev)
        self.burn_penalty = burn_penalty
        self.graph = None
        if capture:
            # launch once outside capture so that every per-kernel attribute
            # and occupancy query is cached, then capture
            self._body(1)
            self.prev.zero_()
            torch.cuda.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._body(self.T)

    def _body(self, T: int):
        for t0 in range(0, T, self.k):
            n = min(self.k, T - t0)
            sl = slice(t0, t0 + n)
            self.sim.step(n, self.drops[sl], self.burning[sl], self.burnt[sl], self.done[sl])
            prev = self.prev[None] if t0 == 0 else self.burning[t0 - 1:t0]
            prevs = torch.cat([prev, self.burning[t0:t0 + n - 1]], 0)
            self.rewards[sl].copy_(reward(self.burning[sl], prevs, self.burn_penalty))
        self.prev.copy_(self.burning[T - 1])

    def run(self):
        """One rollout (graph replay, or eager launches without a graph)."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._body(self.T)
        return self.rewards
