"""The air-tanker agent environment of Section 4 on libjwf (jwf_agent_reset /
jwf_agent_step): N grids stepped together, one agent per grid, everything on
the device.  TankerEnv is the step-by-step interface a policy loop uses;
GraphTankerRollout captures T steps with actions read from a device buffer
(e.g. written by a policy network inside the same graph) as one CUDA graph.
"""
from __future__ import annotations

import torch

from . import jwf


class TankerEnv:
    def __init__(self, sim: jwf.Sim, F0: torch.Tensor, water0: int = 10, obs_k: int = 5,
                 burn_penalty: float = 0.01, random_fire: bool = True):
        self.sim, self.F0 = sim, F0
        self.water0, self.obs_k = int(water0), int(obs_k)
        self.burn_penalty, self.random_fire = float(burn_penalty), bool(random_fire)
        dev = F0.device
        N = sim.N
        self.agent = torch.zeros((N, 3), dtype=torch.int32, device=dev)
        self.obs = torch.zeros((N, self.obs_k, self.obs_k), dtype=torch.uint8, device=dev)
        self.reward = torch.zeros(N, dtype=torch.float32, device=dev)
        self.done = torch.zeros(N, dtype=torch.uint8, device=dev)

    def reset(self) -> torch.Tensor:
        self.sim.load_state(self.F0)
        self.sim.agent_reset(self.agent, self.water0, self.random_fire, self.obs_k, self.obs)
        return self.obs

    def step(self, actions: torch.Tensor):
        """actions int32 [N] -> (obs, reward, done); the tensors are reused
        from step to step."""
        self.sim.agent_step(actions, self.agent, self.water0, self.random_fire, self.burn_penalty, self.reward,
                            self.done, self.obs_k, self.obs)
        return self.obs, self.reward, self.done


class GraphTankerRollout:
    """T agent steps with actions[t] (int32 [T, N], device) as one CUDA graph;
    rewards and done flags are recorded as [T, N].  Capturing runs one
    warm-up step eagerly (reset the env before run())."""

    def __init__(self, env: TankerEnv, actions: torch.Tensor, capture: bool = True):
        self.env, self.actions = env, actions.contiguous()
        T, N = self.actions.shape
        self.T = T
        dev = actions.device
        self.rewards = torch.zeros((T, N), dtype=torch.float32, device=dev)
        self.dones = torch.zeros((T, N), dtype=torch.uint8, device=dev)
        self.graph = None
        if capture:
            self._body(1)
            torch.cuda.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._body(T)

    def _body(self, T: int):
        for t in range(T):
            _, r, d = self.env.step(self.actions[t])
            self.rewards[t].copy_(r)
            self.dones[t].copy_(d)

    def run(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._body(self.T)
        return self.rewards
