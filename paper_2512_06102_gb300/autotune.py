"""Autotuner for the step kernels: block size per size class (resident path),
threads a tile and steps per launch of the tiled path, and steps per launch
for rollouts whose actions are known in advance.

Each candidate is timed with CUDA events on a short probe of the caller's own
workload (the Sim, its initial states and drops); the Sim is restored to the
initial states afterwards.  Choices are cached in a JSON file (path from the
JWF_AUTOTUNE_CACHE environment variable, default ~/.cache/jwf_autotune.json),
keyed by the batch's shape signature, kernel and device name.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import torch

from . import jwf

THREADS = (32, 64, 128, 256, 512, 1024)
TILE_THREADS = (128, 256, 512)
ROUND_STEPS = (4, 8, 16)


def _cache_path() -> str:
    return os.environ.get("JWF_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "jwf_autotune.json"))


def _load_cache() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(cache: dict):
    p = _cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass


def tiled_kernel(kernel: int) -> bool:
    return kernel in (jwf.KERNEL_TILED, jwf.KERNEL_TILED_FUSED)


def signature(sim: jwf.Sim, kernel: int, probe_steps: int) -> str:
    shapes, counts = np.unique(np.stack([sim.H, sim.W], 1), axis=0, return_counts=True)
    h = hashlib.sha256()
    h.update(shapes.tobytes())
    h.update(counts.tobytes())
    dev = torch.cuda.get_device_name(torch.cuda.current_device())
    return f"{dev}|k{kernel}|p{probe_steps}|{h.hexdigest()[:20]}"


def _time(fn, reps: int = 2, prep=None) -> float:
    """Best device time of fn() over reps; prep() (untimed) runs before each."""
    best = float("inf")
    for _ in range(reps):
        if prep is not None:
            prep()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune(sim: jwf.Sim, F0: torch.Tensor, drops: torch.Tensor | None = None, kernel: int = jwf.KERNEL_FUSED,
         probe_steps: int = 32, use_cache: bool = True) -> dict:
    """Pick block sizes per size class (resident path) or steps per launch
    (tiled path) for `sim` stepping from the initial states F0 with `drops`
    ([>= probe_steps, N, 2] or None).  Applies the choice to `sim`, restores
    the initial states and returns the choice."""
    key = signature(sim, kernel, probe_steps)
    cache = _load_cache() if use_cache else {}
    sim.set_kernel(kernel, 0)
    classes = sim.size_classes()
    if key in cache:
        choice = cache[key]
    else:
        dr = None if drops is None else drops[:probe_steps].contiguous()

        def probe():
            sim.load_state(F0)
            sim.step(probe_steps, dr)

        choice = {"class_threads": {}, "round_steps": 16, "tile_threads": 0}
        tiled = kernel in (jwf.KERNEL_TILED, jwf.KERNEL_TILED_FUSED)
        if tiled:
            # the first rounds are dominated by the one-time copies of the
            # tiles without fire; time the probe after probe_steps untimed
            # steps (same drops), when only the fire fronts work
            def warm():
                sim.load_state(F0)
                sim.step(probe_steps, dr)

            def late():
                sim.step(probe_steps, dr)

            best = None
            for th in TILE_THREADS:
                sim.set_kernel(kernel, th)
                for rs in ROUND_STEPS:
                    sim.set_round_steps(rs)
                    t = _time(late, prep=warm)
                    if best is None or t < best[0]:
                        best = (t, rs, th)
            choice["round_steps"] = best[1]
            choice["tile_threads"] = best[2]
        else:
            # coordinate descent over the classes (they run side by side)
            for c in classes:
                best = None
                for th in THREADS:
                    try:
                        sim.set_class_threads(c, th)
                    except jwf.JwfError:
                        continue            # that block size does not fit this class's envs
                    t = _time(probe)
                    if best is None or t < best[0]:
                        best = (t, th)
                choice["class_threads"][str(c)] = best[1]
                sim.set_class_threads(c, best[1])
        if use_cache:
            cache[key] = choice
            _store_cache(cache)
    for c, th in choice.get("class_threads", {}).items():
        if int(c) in classes:
            sim.set_class_threads(int(c), int(th))
    sim.set_kernel(kernel, int(choice.get("tile_threads", 0)) if tiled_kernel(kernel) else 0)
    sim.set_round_steps(int(choice.get("round_steps", 16)))
    sim.load_state(F0)
    torch.cuda.synchronize()
    return choice


def tune_steps_per_launch(sim: jwf.Sim, F0: torch.Tensor, drops: torch.Tensor | None, total_steps: int,
                          candidates=(1, 8, 32, None)) -> int:
    """For actions known in advance: the number of steps per jwf_step call
    (None = all at once) that runs `total_steps` fastest.  Restores F0."""
    best = None
    for k in candidates:
        kk = total_steps if k is None else min(k, total_steps)

        def run():
            sim.load_state(F0)
            for s0 in range(0, total_steps, kk):
                n = min(kk, total_steps - s0)
                sim.step(n, None if drops is None else drops[s0:s0 + n])

        t = _time(run, reps=1)
        if best is None or t < best[0]:
            best = (t, kk)
    sim.load_state(F0)
    return best[1]
