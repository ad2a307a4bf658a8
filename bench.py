#!/usr/bin/env python
"""Benchmark of the JaxWildfire hot path on libjwf (GB300).

One step = one full episode of the batched workload: 4096 grids of 128 x 128
cells (30 m; 11-class fBm landcover, fBm DEM 0-2000 m, per-grid wind, 1-3
fires), reset to the initial fires, the per-grid wind part of Eqs. 1-4, then
200 discrete steps (Section 3 stochastic update, the rates of Eqs. 1-4
evaluated inside the step) with one random 3 x 3 tanker drop per grid per
step and per-step burning/burned counts and done flags.  Metric:
cell-updates/s (grids x cells x steps / time).

The same JSON line also reports the relaxed path (Eqs. 5-10): a forward and
backward pass of 256 grids of 128 x 128 over T = 100 steps (every state kept;
also with sqrt(T) checkpoints), as fwd+bwd cell-steps/s, and the other
workloads (ragged rollout, large maps, the air-tanker scenario).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own batch (weak scaling, no collective in
the data path); rank 0 prints one JSON line.  --impl reference times the CPU
oracle (FP64 table + the plain C simulator), env-parallel over the host cores,
on a sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ENVS, SIDE, EPISODE = 4096, 128, 200
REORDER_STEPS = 12          # the library's default split of a resident launch (jwf_set_reorder_steps)
REL_ENVS, REL_T = 256, 100
RAG_ENVS, RAG_T, RAG_TMAX = 10000, 500, 200
BIG_ENVS, BIG_SIDE, BIG_T = 8, 4096, 1000
TANK_ENVS, TANK_SIDE, TANK_T = 16384, 20, 500
CAL_ENVS, CAL_T, CAL_ITERS, CAL_ITERS_1000 = 256, 100, 40, 2
METRIC = "CA cell-updates/s at 4096x128^2 (200-step episode with tanker drops)"
CPU_SAMPLE_ENVS = 48
REF_PER_CORE = 4            # grids per host process and step of the reference arm
# lane-operation model of the step (instruction counts of the work the model
# requires, independent of how the kernel schedules it): per 32-cell word and
# step, the eight source masks (six funnel shifts, seven ORs) and the state
# update; per Philox4x32-10 block, ten rounds of two wide multiplies and two
# three-input XORs; per draw, the 24-bit conversion and compare; per compared
# pair, the rate of Eqs. 1-4 (double-float slope angle, two exponentials).
OPS_WORD, OPS_PHILOX, OPS_DRAW, OPS_RATE = 20, 40, 4, 140


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-relaxed", action="store_true")
    ap.add_argument("--no-rollout", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-tanker", action="store_true")
    ap.add_argument("--no-calibrate", action="store_true")
    ap.add_argument("--profile", choices=["resident", "relaxed", "tiled", "plain", "prob"], default=None,
                    help="run one small case of a kernel family once (for ncu captures); prints no bench line")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU)
# ---------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class Dist:
    def __init__(self, use_cuda: bool):
        import torch
        self.rank, self.world, self.local = dist_env()
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            backend = "nccl" if use_cuda else "gloo"
            if use_cuda:
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if self.pg is None:
            return x
        import torch
        dev = torch.device("cuda", self.local) if torch.cuda.is_available() else torch.device("cpu")
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class _Nvml:
    """Read-only NVML queries through ctypes (the library ships with the driver):
    the SM clock, its maximum and the active clock event reasons."""
    SM = 1                                   # NVML_CLOCK_SM
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_index: int):
        import ctypes
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        ok = False
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(torch_index).uuid)
            ok = self.lib.nvmlDeviceGetHandleByUUID(("GPU-" + uuid).encode(), ctypes.byref(self.h)) == 0
        except Exception:
            ok = False
        if not ok and self.lib.nvmlDeviceGetHandleByIndex_v2(torch_index, ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = fn or self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def sm(self) -> int:
        v = self.c.c_uint()
        return v.value if self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, self.c.byref(v)) == 0 else -1

    def sm_max(self) -> int:
        v = self.c.c_uint()
        return v.value if self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, self.c.byref(v)) == 0 else -1

    def reasons(self) -> int:
        v = self.c.c_ulonglong()
        return v.value if self.reasons_fn(self.h, self.c.byref(v)) == 0 else 0

    def close(self):
        self.lib.nvmlShutdown()


class Clocks:
    """SM clock and clock event reasons sampled every millisecond (NVML) while
    the timed region runs; only samples between begin() and end() count.
    Falls back to nvidia-smi at 200 ms when NVML cannot be loaded."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.nvml = None
        self.window = [None, None]
        self.halt = threading.Event()

    def start(self):
        try:
            self.nvml = _Nvml(self.index)
            self.th = threading.Thread(target=self._poll, daemon=True)
            self.th.start()
            return
        except (OSError, AttributeError):
            self.nvml = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def begin(self):
        self.window[0] = time.perf_counter()

    def end(self):
        self.window[1] = time.perf_counter()

    def _poll(self):
        while not self.halt.is_set():
            self.rows.append((time.perf_counter(), self.nvml.sm(), self.nvml.reasons()))
            self.halt.wait(0.001)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.nvml is not None:
            self.halt.set()
            self.th.join(timeout=2)
            t0, t1 = self.window
            rows = [r for r in self.rows if (t0 is None or r[0] >= t0) and (t1 is None or r[0] <= t1)]
            sm = [r[1] for r in rows if r[1] > 0]
            reasons = sorted({n for r in rows for bit, n in _Nvml.REASONS.items() if r[2] & bit})
            rec = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.nvml.sm_max(),
                   "reasons": reasons, "samples": len(sm), "source": "NVML, 1 ms"}
            self.nvml.close()
            return rec
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for n, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, 200 ms"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_traffic(name: str, source: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(name)
    if not d:
        return None
    sha = hashlib.sha256(open(os.path.join(ROOT, source), "rb").read()).hexdigest()[:16]
    return d.get("dram_bytes_per_launch") if d.get("source_sha") == sha else None


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_2512_06102_gb300 import build, jwf, scenarios
    from paper_2512_06102_gb300 import relaxed as rlx

    D = Dist(use_cuda=True)
    rank, world = D.rank, D.world
    torch.cuda.set_device(D.local)
    dev = torch.device("cuda", D.local)
    # one build per node (local rank 0); the other ranks wait for it
    if D.local == 0:
        build.build()
    D.barrier()
    if not build.up_to_date():
        raise RuntimeError("libjwf is missing or older than its sources after the local build")

    scn = scenarios.make_scenario(SIDE, SIDE, N=N_ENVS, seed=rank)
    drops = scenarios.drops(EPISODE, scn.H, scn.W, seed=rank)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    cls_d, dem_d, ws_d, wd_d, F0_d, drops_d = (to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir),
                                               to(scn.F0), to(drops))
    sim = jwf.Sim(SIDE, SIDE, n_envs=N_ENVS, n_classes=scenarios.N_CLASSES, seed=1000 + rank)
    sim.set_params(scn.params)
    burning = torch.empty((EPISODE, N_ENVS), dtype=torch.int32, device=dev)
    burnt = torch.empty_like(burning)
    done = torch.empty((EPISODE, N_ENVS), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    ev_k = []

    sim.set_kernel(jwf.KERNEL_FUSED)
    sim.set_reorder_steps(REORDER_STEPS)

    def episode(record=False):
        # reset to the initial fires, (re)build the wind part of Eqs. 1-4, and
        # run the episode; the fused kernel evaluates the ignition probability
        # of every compared (target, source) pair from the terrain
        sim.load_state(F0_d)
        sim.set_terrain(cls_d, dem_d, ws_d, wd_d)
        if record:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        sim.step(EPISODE, drops_d, burning, burnt, done)
        if record:
            b.record(stream)
            ev_k.append((a, b))

    # work of one episode, counted on the device once (the trajectory is
    # deterministic, so every timed episode does the same work)
    counts = torch.zeros(4, dtype=torch.int64, device=dev)
    sim.set_pair_counter(counts)
    episode()
    sim.set_pair_counter(None)
    torch.cuda.synchronize()
    n_pairs, n_blocks, n_burn, n_words = (int(x) for x in counts.tolist())
    active = burning.sum(dtype=torch.int64).item()

    for _ in range(args.warmup):
        episode()
    torch.cuda.synchronize()
    D.barrier()
    clk = Clocks(torch.cuda.current_device())
    clk.start()
    torch.cuda.synchronize()
    D.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk.begin()
    e0.record(stream)
    for _ in range(args.steps):
        episode(record=True)
    e1.record(stream)
    torch.cuda.synchronize()
    clk.end()
    D.barrier()
    t_dev = e0.elapsed_time(e1) / 1e3
    t_kernel = statistics.mean(a.elapsed_time(b) for a, b in ev_k) / 1e3
    clocks = clk.stop()
    t_max = D.max(t_dev)
    cells = N_ENVS * SIDE * SIDE
    units = cells * EPISODE * args.steps
    value = world * units / t_max

    # end to end through the public API with host buffers: inputs copied in
    # from pinned memory and the per-step counts read back, every step.  The
    # initial fires travel 2-bit packed (jwf_load_state_packed), a quarter of
    # the byte-per-cell array.
    P0_d = jwf.pack_states(F0_d)
    host = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            for k, a in (("cls", scn.cls), ("dem", scn.dem), ("ws", scn.wind_speed), ("wd", scn.wind_dir),
                         ("drops", drops))}
    host["P0"] = P0_d.cpu().pin_memory()
    out_h = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory()
             for k, v in (("burning", burning), ("burnt", burnt), ("done", done))}
    dev_in = {"cls": cls_d, "dem": dem_d, "ws": ws_d, "wd": wd_d, "P0": P0_d, "drops": drops_d}
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = sum(v.numel() * v.element_size() for v in out_h.values())

    # two sets of device buffers so that the next episode's inputs are copied
    # in (on a copy stream) while the current episode runs; every episode's
    # copies in and out stay inside the timed region
    s_main = torch.cuda.current_stream()
    s_copy = torch.cuda.Stream()
    sets = [dev_in, {k: torch.empty_like(v) for k, v in dev_in.items()}]
    outs = [(burning, burnt, done), (torch.empty_like(burning), torch.empty_like(burnt), torch.empty_like(done))]
    host_out = [out_h, {k: torch.empty_like(v).pin_memory() for k, v in out_h.items()}]

    def e2e_run(n):
        ev_in = [torch.cuda.Event(), torch.cuda.Event()]
        ev_done = [None, None]
        with torch.cuda.stream(s_copy):
            for k, v in host.items():
                sets[0][k].copy_(v, non_blocking=True)
            ev_in[0].record(s_copy)
        for i in range(n):
            b = i % 2
            if i + 1 < n:
                nb = (i + 1) % 2
                with torch.cuda.stream(s_copy):
                    if ev_done[nb] is not None:
                        s_copy.wait_event(ev_done[nb])      # the set's last episode has finished
                    for k, v in host.items():
                        sets[nb][k].copy_(v, non_blocking=True)
                    ev_in[nb].record(s_copy)
            s_main.wait_event(ev_in[b])
            d = sets[b]
            sim.load_state_packed(d["P0"])
            sim.set_terrain(d["cls"], d["dem"], d["ws"], d["wd"])
            ob = outs[b]
            sim.step(EPISODE, d["drops"], ob[0], ob[1], ob[2])
            ev = torch.cuda.Event()
            ev.record(s_main)
            ev_done[b] = ev
            with torch.cuda.stream(s_copy):
                s_copy.wait_event(ev)
                host_out[b]["burning"].copy_(ob[0], non_blocking=True)
                host_out[b]["burnt"].copy_(ob[1], non_blocking=True)
                host_out[b]["done"].copy_(ob[2], non_blocking=True)
        torch.cuda.synchronize()

    e2e_run(2)
    D.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_run(args.steps)
    torch.cuda.synchronize()
    t_e2e = D.max(time.perf_counter() - t0)
    e2e_value = world * units / t_e2e

    # roofline of the dominant kernel (the resident step launch).  The grid
    # stays in shared memory for the whole episode, so DRAM is not its bound
    # (the byte model below is reported for reference); the bound is
    # instruction issue: the model's lane-operations per launch against
    # SMs x 128 lanes x max SM clock.
    hbm, peak_kind = peaks()
    # an episode is one resident launch, or two with the reorder kernel between them
    split = EPISODE >= 2 * REORDER_STEPS and len(sim.size_classes()) == 1
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz", 2070.0) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 2070.0
    alu_peak = props.multi_processor_count * 128 * sm_mhz * 1e6 / 1e12          # T lane-ops/s
    ops = (OPS_WORD * n_words + OPS_PHILOX * (n_blocks + n_burn) + OPS_DRAW * (n_pairs + n_burn)
           + OPS_RATE * n_pairs)
    alu_ach = ops / t_kernel / 1e12
    b_alg = 2 * cells * EPISODE + 4 * n_pairs + 8 * N_ENVS * EPISODE
    b_min = 2 * cells + 4 * n_pairs + 8 * N_ENVS * EPISODE
    roof = {"bound": "alu", "achieved": round(alu_ach, 3), "peak": round(alu_peak, 2), "unit": "T lane-ops/s",
            "frac": round(alu_ach / alu_peak, 4),
            "peak_source": f"{props.multi_processor_count} SMs x 128 lanes x {sm_mhz:.0f} MHz",
            "traffic": kernel_traffic("k_step_resident", "paper_2512_06102_gb300/csrc/k_resident.cu"),
            "kernel": "k_step_resident (fused)" + (" x2 + k_reorder (one episode)" if split else ""),
            "kernel_ms": round(t_kernel * 1e3, 3),
            "ops_model": (f"{OPS_WORD}/bit-plane word-step + {OPS_PHILOX}/Philox4x32-10 block + "
                          f"{OPS_DRAW}/draw compare + {OPS_RATE}/pair rate evaluation (Eqs. 1-4)"),
            "ops_per_launch": ops,
            "work": {"pairs": n_pairs, "philox_blocks_candidates": n_blocks, "burning_draws": n_burn,
                     "word_steps": n_words, "burning_cell_steps": active},
            "hbm_byte_model": {"bytes_per_launch": b_alg, "model": "2 B/cell-update + 4 B/compared pair + 8 B/env-step",
                               "achieved_gbs": round(b_alg / t_kernel / 1e9, 1), "peak_gbs": hbm,
                               "peak_source": peak_kind, "frac": round(b_alg / t_kernel / 1e9 / hbm, 4),
                               "min_bytes_per_launch": b_min,
                               "min_bytes_frac": round(b_min / t_kernel / 1e9 / hbm, 4)}}
    # comparators on the same workload: the table path (table kernel + resident
    # step reading q) and the plain one-launch-per-step path
    def timed(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    def table_episode():
        sim.load_state(F0_d)
        sim.precompute_probs(cls_d, dem_d, ws_d, wd_d)
        sim.step(EPISODE, drops_d, burning, burnt, done)

    sim.set_kernel(jwf.KERNEL_RESIDENT)
    table_episode()
    t_table = timed(table_episode)
    sim.set_kernel(jwf.KERNEL_PLAIN)
    t_plain = timed(table_episode)
    # the same episode with the wind changing every step (a [200][N] series;
    # the fused kernel evaluates each step's rates, no table to rebuild)
    gw = torch.Generator(device=dev).manual_seed(11)
    ws_ser = torch.rand((EPISODE, N_ENVS), device=dev, generator=gw) * 10.0
    wd_ser = torch.rand((EPISODE, N_ENVS), device=dev, generator=gw) * (2.0 * np.pi)
    sim.set_kernel(jwf.KERNEL_FUSED)
    sim.set_wind_series(ws_ser, wd_ser)
    episode()
    t_series = timed(episode)
    sim.set_wind_series(None)
    comparators = {"table_resident_ms_per_step": round(t_table * 1e3, 3),
                   "plain_one_launch_per_step_ms_per_step": round(t_plain * 1e3, 3),
                   "speedup_vs_plain": round(t_plain / (t_max / args.steps), 2),
                   "speedup_vs_table_resident": round(t_table / (t_max / args.steps), 2),
                   "wind_series_ms_per_step": round(t_series * 1e3, 3)}
    sim.close()
    del sim

    # the single-environment workload: one 64 x 64 grid, one fuel class, flat,
    # no wind, a fire at the centre, 100 steps (latency-bound: time only)
    one = scenarios.plain_single_env(64, 64)
    sim1 = jwf.Sim(64, 64, n_envs=1, n_classes=1, seed=0)
    sim1.set_params(one.params)
    o_to = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (one.cls, one.dem, one.wind_speed,
                                                                         one.wind_dir, one.F0)]
    sim1.set_terrain(*o_to[:4])
    sim1.set_kernel(jwf.KERNEL_FUSED)

    def single():
        sim1.load_state(o_to[4])
        sim1.step(100)

    single()
    t_single = min(timed(single) for _ in range(5))
    sim1.close()
    comparators["single_env_64x64_100_steps_ms"] = round(t_single * 1e3, 3)

    rel = None
    if not args.no_relaxed:
        rel = bench_relaxed(args, D, dev, rank)
    rag = None
    if not args.no_rollout:
        rag = bench_rollout(args, D, dev, rank)
    big = None
    if not args.no_large:
        big = bench_large(args, D, dev, rank)
    tank = None
    if not args.no_tanker:
        tank = bench_tanker(args, D, dev, rank)
    cal = None
    if not args.no_calibrate:
        cal = bench_calibrate(args, D, dev, rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(scn, drops)
        cpu["parallel"] = cpu_parallel(scn, drops)
        cpu["relaxed"] = cpu_relaxed()
        cpu["large"] = cpu_large()

    line = {"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded fBm landcover/DEM stand-ins for WorldCover/GLO-30)",
            "config": {"workload": f"batched: {N_ENVS} grids x {SIDE}x{SIDE}, {EPISODE}-step episode, 3x3 drop/step",
                       "global_batch": N_ENVS * world, "grid": [SIDE, SIDE], "steps_per_episode": EPISODE,
                       "parallelism": f"replicas x{world} (independent grid shards)",
                       "l2": "inputs larger than L2 (landcover + DEM 335 MB and the 67 MB states read every episode)"},
            "env_steps_per_s": world * N_ENVS * EPISODE * args.steps / t_max,
            "roofline": roof,
            "comparators": comparators,
            "e2e": {"value": e2e_value, "unit": "cell-updates/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": (5 if split else 3) * args.steps,
            "clocks": clocks}
    if rel is not None:
        line["relaxed"] = rel
    if rag is not None:
        line["rollout"] = rag
    if big is not None:
        line["large"] = big
    if tank is not None:
        line["tanker"] = tank
    if cal is not None:
        line["calibrate"] = cal
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    D.close()


def bench_relaxed(args, D, dev, rank):
    """fwd+bwd of T relaxed steps on 256 x 128^2: tiled kernels with every state
    kept (the default policy when the states fit), then sqrt(T) checkpoints,
    then the plain kernels (one thread per cell, two-pass adjoint) with sqrt(T)
    checkpoints as the comparator; T = 1000 with sqrt(T) checkpoints once."""
    import torch

    from paper_2512_06102_gb300 import jwf, scenarios
    from paper_2512_06102_gb300 import relaxed as rlx

    scn = scenarios.make_scenario(SIDE, SIDE, N=REL_ENVS, seed=100 + rank)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    scene = (to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    sim = jwf.Sim(SIDE, SIDE, n_envs=REL_ENVS, n_classes=scenarios.N_CLASSES, keep_rates=True)
    p = scn.params
    theta0 = torch.tensor([p.p_base, p.alpha_w1, p.alpha_w2, p.alpha_s, p.alpha_gamma, p.p_continue]
                          + list(p.mu_veg) + list(p.mu_den), dtype=torch.float64)
    pb0 = (to(scn.F0) == 2).float()
    pu0 = 1.0 - pb0
    target = torch.rand(pu0.shape, device=dev, generator=torch.Generator(device=dev).manual_seed(7))
    stream = torch.cuda.current_stream()
    cells = REL_ENVS * SIDE * SIDE

    def fwd_bwd(T, ckpt):
        th = theta0.clone().requires_grad_(True)
        pu = pu0.clone().requires_grad_(True)
        pb = pb0.clone().requires_grad_(True)
        ou, ob = rlx.rollout(th, pu, pb, sim, scene, T, ckpt_every=ckpt)
        loss = ((ou - target) ** 2).mean() + ob.mean()
        loss.backward()
        return th.grad

    clock_rec = {}

    def timed(T, ckpt, steps, warmup):
        for _ in range(max(1, warmup)):
            fwd_bwd(T, ckpt)
        torch.cuda.synchronize()
        D.barrier()
        clk = Clocks(torch.cuda.current_device())
        clk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk.begin()
        e0.record(stream)
        for _ in range(steps):
            fwd_bwd(T, ckpt)
        e1.record(stream)
        torch.cuda.synchronize()
        clk.end()
        clock_rec.setdefault((T, ckpt), clk.stop())
        D.barrier()
        return D.max(e0.elapsed_time(e1) / 1e3) / steps

    # the two dominant kernels, timed in isolation over n launches
    def time_kernels(n=20):
        sim.set_params(rlx.theta_to_params(theta0, sim.n_classes))
        sim.precompute_probs(*scene)
        bufs = [(pu0.clone(), pb0.clone()), (torch.empty_like(pu0), torch.empty_like(pb0))]
        g = [(torch.randn_like(pu0), torch.randn_like(pu0)), (torch.empty_like(pu0), torch.empty_like(pu0))]
        glam = torch.empty_like(pu0)
        gpc = torch.zeros(1, dtype=torch.float64, device=dev)
        out = {}
        two = (torch.empty((2,) + pu0.shape, device=dev), torch.empty((2,) + pu0.shape, device=dev))
        PU2, PB2 = torch.stack([pu0, pu0]), torch.stack([pb0, pb0])
        glam2 = torch.empty((2,) + pu0.shape, device=dev)
        glam16 = torch.randn((16,) + pu0.shape, device=dev)
        pb16 = torch.rand((16,) + pu0.shape, device=dev)
        gr = torch.zeros((cells, 8), device=dev)
        for name in ("fwd", "fwd2", "bwd", "bwd2", "acc16"):
            for i in range(n + 1):
                if i == 1:
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                src, dst = bufs[i % 2], bufs[(i + 1) % 2]
                if name == "fwd":
                    sim.relaxed_fwd(src[0], src[1], None, dst[0], dst[1])
                elif name == "fwd2":
                    # two steps in one pass (the rollout's forward)
                    sim.relaxed_fwd_steps(bufs[0][0], bufs[0][1], two[0], two[1])
                elif name == "bwd2":
                    # two adjoint steps in one pass (the rollout's backward)
                    gs, gd = g[i % 2], g[(i + 1) % 2]
                    sim.relaxed_bwd_steps(PU2, PB2, gs[0], gs[1], gd[0], gd[1], glam=glam2, gpc=gpc)
                elif name == "acc16":
                    # the rate adjoint of a 16-step block
                    sim.rates_accumulate(glam16, pb16, gr)
                else:
                    gs, gd = g[i % 2], g[(i + 1) % 2]
                    sim.relaxed_bwd(bufs[0][0], bufs[0][1], gs[0], gs[1], None, gd[0], gd[1], glam, gpc)
            e1.record(stream)
            torch.cuda.synchronize()
            out[name] = e0.elapsed_time(e1) / 1e3 / n
        return out

    sim.set_relaxed_kernel(jwf.RELAXED_TILED)
    keep_all = rlx.resolve_ckpt(REL_T, cells, None, dev)
    t_keep = timed(REL_T, None, args.steps, args.warmup)
    t_sqrt = timed(REL_T, "sqrt", args.steps, args.warmup)
    t_1000 = timed(1000, "sqrt", 1, 1)
    k_tiled = time_kernels()
    sim.set_relaxed_kernel(jwf.RELAXED_PLAIN)
    t_plain = timed(REL_T, "sqrt", args.steps, args.warmup)
    k_plain = time_kernels()
    sim.set_relaxed_kernel(jwf.RELAXED_TILED)
    hbm, peak_kind = peaks()
    fwd1_b, fwd_b, bwd1_b, bwd_b, acc_b = 48, 28, 60, 36, 12
    ach_b = 2 * bwd_b * cells / k_tiled["bwd2"] / 1e9
    ach_b1 = bwd1_b * cells / k_tiled["bwd"] / 1e9
    ach_acc = 16 * acc_b * cells / k_tiled["acc16"] / 1e9
    ach_f = fwd1_b * cells / k_tiled["fwd"] / 1e9
    ach_f2 = 2 * fwd_b * cells / k_tiled["fwd2"] / 1e9
    rate = D.world * cells * REL_T / t_keep
    sim.close()
    return {"metric": "fwd+bwd cell-steps/s at 256x128^2, T=100",
            "value": rate, "unit": "fwd+bwd cell-steps/s",
            "ms_per_step": t_keep * 1e3, "dtype": "f32", "clocks": clock_rec.get((REL_T, None)),
            "memory_policy": "every state kept" if keep_all == 0 else "sqrt(T) checkpoints",
            "path_bytes_model": f"{fwd_b + bwd_b + acc_b} B/cell-step ({fwd_b} two-step fwd + {bwd_b} two-step "
                                f"fused adjoint + {acc_b} rate-adjoint accumulation)",
            "path_gbs": round((fwd_b + bwd_b + acc_b) * rate / D.world / 1e9, 1),
            "path_frac": round((fwd_b + bwd_b + acc_b) * rate / D.world / 1e9 / hbm, 4),
            "roofline": {"bound": "hbm", "achieved": round(ach_b, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(ach_b / hbm, 4), "peak_source": peak_kind,
                         "traffic": kernel_traffic("k_relaxed_bwd_sweep2", "paper_2512_06102_gb300/csrc/k_relaxed.cu"),
                         "kernel": "k_relaxed_bwd_sweep2 (two adjoint steps a pass)",
                         "kernel_us": round(k_tiled["bwd2"] * 1e6, 2),
                         "bytes_model": "36 B/cell-step (per two steps: 32 B rates, 16 B states, 8 B adjoint in, "
                                        "8 B adjoint out, 8 B glam)"},
            "roofline_bwd1": {"bound": "hbm", "achieved": round(ach_b1, 1), "peak": hbm, "unit": "GB/s",
                              "frac": round(ach_b1 / hbm, 4), "kernel": "k_relaxed_bwd_sweep (one step, "
                              "jwf_step_relaxed_bwd)", "kernel_us": round(k_tiled["bwd"] * 1e6, 2),
                              "bytes_model": "60 B/cell-step (32 B rates, 8 B state, 8 B adjoint in, 8 B adjoint "
                                             "out, 4 B glam)"},
            "roofline_acc": {"bound": "hbm", "achieved": round(ach_acc, 1), "peak": hbm, "unit": "GB/s",
                             "frac": round(ach_acc / hbm, 4), "kernel": "k_rates_accumulate (16-step block)",
                             "kernel_us": round(k_tiled["acc16"] * 1e6, 2),
                             "bytes_model": "12 B/cell-step (4 B glam, 4 B p_burn; 64 B rate adjoint read and "
                                            "written per 16 steps)"},
            "roofline_fwd": {"bound": "hbm", "achieved": round(ach_f, 1), "peak": hbm, "unit": "GB/s",
                             "frac": round(ach_f / hbm, 4), "kernel": "k_relaxed_fwd_tiled",
                             "kernel_us": round(k_tiled["fwd"] * 1e6, 2),
                             "bytes_model": "48 B/cell-step (8 B state in, 32 B rates, 8 B state out)"},
            "roofline_fwd2": {"bound": "hbm", "achieved": round(ach_f2, 1), "peak": hbm, "unit": "GB/s",
                              "frac": round(ach_f2 / hbm, 4), "kernel": "k_relaxed_fwd2_tiled (two steps a pass)",
                              "kernel_us": round(k_tiled["fwd2"] * 1e6, 2),
                              "bytes_model": "28 B/cell-step (per two steps: 8 B state in, 32 B rates, 16 B "
                                             "states out)"},
            "sqrt_checkpoints": {"ms_per_step": round(t_sqrt * 1e3, 3),
                                 "value": D.world * cells * REL_T / t_sqrt},
            "T1000_sqrt_checkpoints": {"ms_per_step": round(t_1000 * 1e3, 3),
                                       "value": D.world * cells * 1000 / t_1000},
            "comparators": {"plain_kernels_sqrt_ms_per_step": round(t_plain * 1e3, 3),
                            "plain_fwd_us": round(k_plain["fwd"] * 1e6, 2),
                            "plain_bwd_pair_us": round(k_plain["bwd"] * 1e6, 2),
                            "speedup_vs_plain": round(t_plain / t_keep, 2),
                            "speedup_vs_plain_same_checkpoints": round(t_plain / t_sqrt, 2),
                            "adjoint_speedup_vs_unfused_pair": round(k_plain["bwd"] / k_tiled["bwd"], 2)}}


def bench_calibrate(args, D, dev, rank):
    """Gradient-based calibration (Section 4) at the differentiation
    workload's size: 256 grids of 128 x 128, targets = burn maps of the
    stochastic step (mean over 5 seeds) from hidden parameters (the defaults
    with p_base and the wind and slope coefficients scaled by U(0.7, 1.3) and
    the burnable classes' mu_veg shifted by U(-0.1, 0.1), seeded), Adam on the
    relaxed rollout from the defaults (T = 100, every state kept; the default
    free set: p_base, alpha_w1, alpha_w2, alpha_s and mu_veg).  Reports fit
    iterations/s (forward, backward, loss and update, host included), the loss
    and the fitted, hidden and starting coefficients; then a few iterations at
    T = 1000 with sqrt(T) checkpoints."""
    import time

    import torch

    from paper_2512_06102_gb300 import calibrate, jwf, scenarios

    scn = scenarios.make_scenario(SIDE, SIDE, N=CAL_ENVS, seed=300 + rank)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    scene = (to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    F0 = to(scn.F0)
    C = scenarios.N_CLASSES
    rng = np.random.default_rng(301 + rank)
    truth = scenarios.Params()
    for name in ("p_base", "alpha_w1", "alpha_w2", "alpha_s"):
        setattr(truth, name, float(getattr(truth, name)) * float(rng.uniform(0.7, 1.3)))
    burnable = scenarios.burnable_classes(truth.mu_den)
    mv = np.array(truth.mu_veg, np.float32)
    mv[burnable] += rng.uniform(-0.1, 0.1, size=int(np.sum(burnable))).astype(np.float32)
    truth.mu_veg = mv
    target = calibrate.burn_maps(SIDE, SIDE, CAL_ENVS, truth, scene, F0, CAL_T)
    start = calibrate.theta_of(scenarios.Params(), C)
    sim = jwf.Sim(SIDE, SIDE, n_envs=CAL_ENVS, n_classes=C, keep_rates=True)
    sim.set_params(scenarios.Params())

    def run(T, iters, ckpt=None):
        torch.cuda.synchronize()
        D.barrier()
        t0 = time.perf_counter()
        th, ls = calibrate.fit(sim, scene, F0, target, start, T, iters=iters, ckpt_every=ckpt)
        torch.cuda.synchronize()
        return D.max(time.perf_counter() - t0), th, ls

    run(CAL_T, 2)                                   # warm-up
    t_fit, theta, losses = run(CAL_T, CAL_ITERS)
    t_1000, _, losses_1000 = run(1000, CAL_ITERS_1000, "sqrt")
    # no model mismatch: targets from the relaxed rollout itself with the
    # hidden coefficients, the four coefficients free
    from paper_2512_06102_gb300 import relaxed as rlx
    pb0 = (F0 == 2).float()
    with torch.no_grad():
        ou, _ = rlx.rollout(calibrate.theta_of(truth, C), 1.0 - pb0, pb0, sim, scene, CAL_T)
    rtarget = (1.0 - ou).clamp(0.0, 1.0)
    free4 = torch.zeros_like(start)
    free4[0:4] = 1.0
    theta_r, losses_r = calibrate.fit(sim, scene, F0, rtarget, start, CAL_T, iters=3 * CAL_ITERS, free=free4)
    with torch.no_grad():
        floor = float(torch.nn.functional.binary_cross_entropy(rtarget, rtarget))
    sim.close()
    names = ("p_base", "alpha_w1", "alpha_w2", "alpha_s")
    coef = {n: {"start": round(float(start[i]), 5), "hidden": round(float(getattr(truth, n)), 5),
                "fitted": round(float(theta[i]), 5)} for i, n in enumerate(names)}
    return {"metric": "calibration fit iterations/s at 256x128^2, T=100 (Adam on the relaxed rollout)",
            "value": CAL_ITERS / t_fit, "unit": "iterations/s", "iterations": CAL_ITERS,
            "ms_per_iteration": round(t_fit / CAL_ITERS * 1e3, 3),
            "fwd_bwd_cell_steps_per_s": D.world * CAL_ENVS * SIDE * SIDE * CAL_T * CAL_ITERS / t_fit,
            "loss_first": round(losses[0], 6), "loss_last": round(losses[-1], 6),
            "target_mean_burned": round(float(target.mean()), 5), "coefficients": coef,
            "mu_veg_fitted_minus_hidden_max_abs": round(float(np.max(np.abs(
                theta[6:6 + C].numpy()[burnable] - np.asarray(truth.mu_veg, np.float64)[burnable]))), 5),
            "relaxed_targets": {"iterations": 3 * CAL_ITERS, "loss_first": round(losses_r[0], 6),
                                "loss_last": round(losses_r[-1], 6), "loss_floor": round(floor, 6),
                                "coefficients": {n: {"start": round(float(start[i]), 5),
                                                     "hidden": round(float(getattr(truth, n)), 5),
                                                     "fitted": round(float(theta_r[i]), 5)}
                                                 for i, n in enumerate(names)}},
            "T1000_sqrt_checkpoints": {"iterations": CAL_ITERS_1000,
                                       "ms_per_iteration": round(t_1000 / CAL_ITERS_1000 * 1e3, 3),
                                       "loss_first": round(losses_1000[0], 6)},
            "note": "targets come from the stochastic step; the mean-field relaxed model is not its multi-step "
                    "expectation, so the fitted coefficients need not equal the hidden ones"}


def bench_large(args, D, dev, rank):
    """8 grids of 4096 x 4096, one 1000-step episode with a random 3x3 drop per
    grid and step, on the tiled temporally blocked path: rates evaluated per
    compared pair (no table), and the table variant with its table build
    inside the timed region; the plain one-launch-per-step path over 200
    steps as the comparator."""
    import torch

    from paper_2512_06102_gb300 import autotune, jwf, scenarios

    scn = scenarios.make_scenario(BIG_SIDE, BIG_SIDE, N=BIG_ENVS, seed=200 + rank)
    drops = scenarios.drops(BIG_T, scn.H, scn.W, seed=200 + rank)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    scene = (to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    F0, dr = to(scn.F0), to(drops)
    sim = jwf.Sim(BIG_SIDE, BIG_SIDE, n_envs=BIG_ENVS, n_classes=scenarios.N_CLASSES, seed=rank)
    sim.set_params(scn.params)
    sim.set_terrain(*scene)
    stream = torch.cuda.current_stream()
    cells = BIG_ENVS * BIG_SIDE * BIG_SIDE

    clock_rec = {}

    def timed(fn, reps):
        best = float("inf")
        clk = Clocks(torch.cuda.current_device())
        clk.start()
        for _ in range(reps):
            sim.load_state(F0)
            torch.cuda.synchronize()
            D.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if clk.window[0] is None:
                clk.begin()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            clk.end()
            best = min(best, D.max(e0.elapsed_time(e1) / 1e3))
        clock_rec[best] = clk.stop()
        return best

    choice = autotune.tune(sim, F0, dr, kernel=jwf.KERNEL_TILED_FUSED, probe_steps=256, use_cache=False)
    th = int(choice.get("tile_threads", 0))
    sim.set_kernel(jwf.KERNEL_TILED_FUSED, th)
    t_fused = timed(lambda: sim.step(BIG_T, dr), max(2, args.steps))
    tma = sim.tile_copy()
    t_loads = None
    if tma:
        # the same episode with the regions staged by plain 128-bit loads
        sim.set_tile_copy(False)
        t_loads = timed(lambda: sim.step(BIG_T, dr), max(2, args.steps))
        sim.set_tile_copy(True)
    cnt = torch.zeros(4, dtype=torch.int64, device=dev)
    sim.set_pair_counter(cnt)
    sim.load_state(F0)
    sim.step(BIG_T, dr)
    sim.set_pair_counter(None)
    torch.cuda.synchronize()
    pairs, blocks, draws, words = [int(x) for x in cnt.tolist()]
    sim.set_kernel(jwf.KERNEL_TILED, th)

    def table_episode():
        sim.precompute_probs(*scene)
        sim.step(BIG_T, dr)

    t_table = timed(table_episode, max(2, args.steps))
    # the states 2-bit packed at the boundary: the initial fires in and the
    # final state out (a quarter of the bytes; inside, the kernels keep one
    # byte a cell), and the same episode run from the packed initial state
    sim.set_kernel(jwf.KERNEL_TILED_FUSED, th)
    P0 = jwf.pack_states(F0)
    Pout = torch.zeros_like(P0)

    def packed_io():
        sim.load_state_packed(P0)
        sim.state_packed(Pout)

    F0u = torch.empty_like(F0)
    t_pack = timed(lambda: jwf.pack_states(F0, P0), 5)
    t_unpack = timed(lambda: jwf.unpack_states(P0, cells, F0u), 5)
    t_io_packed = timed(packed_io, 5)
    t_io_u8 = timed(lambda: (sim.load_state(F0), sim.state_views()[0].clone()), 5)

    def packed_episode():
        sim.load_state_packed(P0)
        sim.step(BIG_T, dr)
        sim.state_packed(Pout)

    t_packed_ep = timed(packed_episode, max(2, args.steps))
    sim.set_kernel(jwf.KERNEL_PLAIN)
    t_plain200 = timed(lambda: sim.step(200, dr[:200]), 1)
    sim.close()
    best = min(t_fused, t_table)
    ops = OPS_WORD * words + OPS_PHILOX * (blocks + draws) + OPS_DRAW * (pairs + draws) + OPS_RATE * pairs
    peak_ops = 152 * 128 * 2.07e9 / 1e12
    return {"metric": "CA cell-updates/s at 8x4096^2 (1000-step episode with tanker drops)",
            "value": D.world * cells * BIG_T / best, "unit": "cell-updates/s", "ms_per_episode": round(best * 1e3, 3),
            "clocks": clock_rec.get(best),
            "kernel": "tiled table (table build included)" if t_table <= t_fused else "tiled fused",
            "fused_ms": round(t_fused * 1e3, 3), "table_with_build_ms": round(t_table * 1e3, 3),
            "round_steps": choice.get("round_steps"), "tile_threads": th,
            "tile_copy": "tma" if tma else "loads",
            "fused_loads_ms": None if t_loads is None else round(t_loads * 1e3, 3),
            "touched": {"word_steps": words, "cell_steps_scanned": 32 * words,
                        "fraction_of_cell_steps": round(32 * words / (cells * BIG_T), 4),
                        "per_touched_cell_rate": 32 * words / t_fused},
            "roofline_fused": {"bound": "alu", "achieved": round(ops / t_fused / 1e12, 3), "peak": round(peak_ops, 2),
                               "unit": "T lane-ops/s", "frac": round(ops / t_fused / 1e12 / peak_ops, 4),
                               "work": {"pairs": pairs, "philox_blocks_candidates": blocks, "burning_draws": draws,
                                        "word_steps": words}},
            "packed_2bit": {"bytes_per_state": int(P0.numel()), "u8_bytes_per_state": cells,
                            "pack_ms": round(t_pack * 1e3, 3), "unpack_ms": round(t_unpack * 1e3, 3),
                            "load_and_read_packed_ms": round(t_io_packed * 1e3, 3),
                            "load_and_read_u8_ms": round(t_io_u8 * 1e3, 3),
                            "episode_packed_in_out_ms": round(t_packed_ep * 1e3, 3),
                            "note": "states travel 2-bit packed at the boundary; the tiled kernel keeps one byte a "
                                    "cell inside (its region copies are a small share of the episode)"},
            "comparators": {"plain_one_launch_per_step_ms_per_1000": round(t_plain200 * 5e3, 1),
                            "speedup_vs_plain": round(t_plain200 * 5 / best, 2)}}


def bench_tanker(args, D, dev, rank):
    """The air-tanker agent scenario of Section 4: 16,384 grids of 20 x 20, one
    agent each (move + valve, 10 units of water, 5 x 5 egocentric window),
    500 agent steps with random actions and auto-reset (random agent position
    and ignition every episode, episode limit 100), as one CUDA graph; eager
    steps and the plain one-launch-per-step kernel as comparators."""
    import torch

    from paper_2512_06102_gb300 import jwf, scenarios, tanker

    scn = scenarios.make_scenario(TANK_SIDE, TANK_SIDE, N=TANK_ENVS, seed=300 + rank)
    F0 = scn.F0.copy()
    F0[F0 == 2] = 1
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    acts = torch.randint(0, 10, (TANK_T, TANK_ENVS), dtype=torch.int32, device=dev,
                         generator=torch.Generator(device=dev).manual_seed(5))
    stream = torch.cuda.current_stream()

    def run(kernel, graph):
        sim = jwf.Sim(TANK_SIDE, TANK_SIDE, n_envs=TANK_ENVS, n_classes=scenarios.N_CLASSES, seed=rank,
                      auto_reset=True, t_max=100)
        sim.set_params(scn.params)
        sim.set_terrain(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
        if kernel == jwf.KERNEL_PLAIN:
            sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
        sim.set_kernel(kernel)
        env = tanker.TankerEnv(sim, to(F0), water0=10, obs_k=5, burn_penalty=0.01, random_fire=True)
        env.reset()
        g = tanker.GraphTankerRollout(env, acts, capture=graph)
        best = float("inf")
        for _ in range(max(1, args.warmup) + 2):
            env.reset()
            torch.cuda.synchronize()
            D.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rw = g.run()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, D.max(e0.elapsed_time(e1) / 1e3))
        ret = float(rw.sum().item()) / TANK_ENVS
        episodes = int(g.dones.sum().item())
        sim.close()
        return best, ret, episodes

    t_graph, ret, episodes = run(jwf.KERNEL_FUSED, True)
    t_eager, _, _ = run(jwf.KERNEL_FUSED, False)
    t_plain, _, _ = run(jwf.KERNEL_PLAIN, True)
    return {"metric": "agent env-steps/s, 16384 x 20^2 tanker scenario, 500 steps, auto-reset (one CUDA graph)",
            "value": D.world * TANK_ENVS * TANK_T / t_graph, "unit": "env-steps/s",
            "ms_per_rollout": round(t_graph * 1e3, 3), "launches_per_step": 1,
            "episodes_finished": episodes, "mean_return_random_policy": round(ret, 3),
            "comparators": {"eager_ms": round(t_eager * 1e3, 3), "plain_kernel_graph_ms": round(t_plain * 1e3, 3),
                            "speedup_vs_eager": round(t_eager / t_graph, 2),
                            "speedup_vs_plain": round(t_plain / t_graph, 2)}}


def bench_rollout(args, D, dev, rank):
    """10,000 grids, side log-uniform in [32, 512], 500-step RL rollout with a
    random 3x3 drop per grid and step, auto-reset (episode limit 200), one CUDA
    graph; steps per launch and block sizes from the autotuner."""
    import torch

    from paper_2512_06102_gb300 import autotune, jwf, rollout, scenarios

    sides = scenarios.ragged_sides(RAG_ENVS, 32, 512, seed=7 + rank)
    scn = scenarios.make_scenario(sides, sides, seed=7 + rank)
    drops = scenarios.drops(RAG_T, scn.H, scn.W, seed=7 + rank)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    terrain = (to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
    F0, dr = to(scn.F0), to(drops)
    cells = int(scn.cls.size)
    sim = jwf.Sim(scn.H, scn.W, n_classes=scenarios.N_CLASSES, seed=2000 + rank, t_max=RAG_TMAX, auto_reset=True)
    sim.set_params(scn.params)
    sim.set_kernel(jwf.KERNEL_FUSED)
    sim.set_terrain(*terrain)
    choice = autotune.tune(sim, F0, dr, kernel=jwf.KERNEL_FUSED, probe_steps=16, use_cache=False)
    k_best = autotune.tune_steps_per_launch(sim, F0, dr, RAG_T, candidates=(64, 125, 250, None))

    def timed(fn, reps=1):
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3
            best = t if best is None else min(best, t)
        return best

    res = {}
    for k in sorted({1, k_best}):
        g = rollout.GraphRollout(sim, RAG_T, dr, steps_per_launch=k)
        sim.load_state(F0)
        g.run()
        D.barrier()
        t = timed(lambda: (sim.load_state(F0), g.run()), reps=max(1, min(args.steps, 3)))
        res[k] = D.max(t)
        del g
    k_use = min(res, key=res.get)
    t_graph = res[k_use]
    # the work of the rollout, counted on the device on one eager pass (the
    # trajectory is deterministic: the timed graph does the same work)
    cnt = torch.zeros(4, dtype=torch.int64, device=dev)
    counted = rollout.GraphRollout(sim, RAG_T, dr, capture=False, steps_per_launch=k_use)
    sim.set_pair_counter(cnt)
    sim.load_state(F0)
    counted.run()
    sim.set_pair_counter(None)
    torch.cuda.synchronize()
    pairs, blocks, draws, words = (int(x) for x in cnt.tolist())
    del counted
    ops = OPS_WORD * words + OPS_PHILOX * (blocks + draws) + OPS_DRAW * (pairs + draws) + OPS_RATE * pairs
    props = torch.cuda.get_device_properties(dev)
    alu_peak = props.multi_processor_count * 128 * 2.07e9 / 1e12
    eager = rollout.GraphRollout(sim, RAG_T, dr, capture=False, steps_per_launch=1)
    t_eager = timed(lambda: (sim.load_state(F0), eager.run()))
    # plain one-launch-per-step path on the same rollout (table built first)
    sim.precompute_probs(*terrain)
    sim.set_kernel(jwf.KERNEL_PLAIN)
    plain = rollout.GraphRollout(sim, RAG_T, dr, capture=False, steps_per_launch=1)
    t_plain = timed(lambda: (sim.load_state(F0), plain.run()))
    sim.close()
    world = D.world
    return {"metric": "env-steps/s, 10000 ragged grids (side log-uniform 32..512), 500-step rollout, auto-reset",
            "value": world * RAG_ENVS * RAG_T / t_graph, "unit": "env-steps/s",
            "cell_updates_per_s": world * cells * RAG_T / t_graph, "cells": cells,
            "ms_per_rollout": round(t_graph * 1e3, 3), "steps_per_launch": k_use,
            "graph_ms_by_steps_per_launch": {str(k): round(v * 1e3, 3) for k, v in res.items()},
            "autotune": choice,
            "roofline": {"bound": "alu", "achieved": round(ops / t_graph / 1e12, 3), "peak": round(alu_peak, 2),
                         "unit": "T lane-ops/s", "frac": round(ops / t_graph / 1e12 / alu_peak, 4), "traffic": None,
                         "kernel": "k_step_resident (fused), four size classes on forked streams, whole rollout",
                         "work": {"pairs": pairs, "philox_blocks_candidates": blocks, "burning_draws": draws,
                                  "word_steps": words}},
            "comparators": {"eager_one_step_launches_ms": round(t_eager * 1e3, 3),
                            "plain_one_launch_per_step_ms": round(t_plain * 1e3, 3),
                            "speedup_vs_plain": round(t_plain / t_graph, 2),
                            "speedup_vs_eager": round(t_eager / t_graph, 2)}}


# ---------------------------------------------------------------------------
# CPU oracle timing (rank 0, N = 1)
# ---------------------------------------------------------------------------
def oracle_episode(scn, drops, envs):
    """The oracle on grids `envs` of the batch: FP64 table + C rollout."""
    import torch

    from oracle import discrete, prob
    p = scn.params.as_dict()
    q = []
    for e in envs:
        q32, _, _, _ = prob.table_f32(scn.env(e, scn.cls)[None], scn.env(e, scn.dem)[None],
                                      scn.wind_speed[e:e + 1], scn.wind_dir[e:e + 1], p, 30.0)
        q.append(q32.reshape(-1, 8))
    n = len(envs)
    F0 = np.concatenate([scn.env(e, scn.F0).reshape(-1) for e in envs])
    ro = discrete.Rollout(np.full(n, SIDE), np.full(n, SIDE), F0, np.concatenate(q), scn.params.p_continue,
                          seed=1000, env_ids=np.asarray(envs, np.int32))
    ro.step(EPISODE, np.ascontiguousarray(drops[:, envs]))


def cpu_baseline(scn, drops, n_envs=CPU_SAMPLE_ENVS, reps=1):
    import torch
    torch.set_num_threads(1)
    envs = list(range(n_envs))
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle_episode(scn, drops, envs)
    dt = time.perf_counter() - t0
    return {"value": reps * n_envs * SIDE * SIDE * EPISODE / dt, "unit": "cell-updates/s", "cores": 1,
            "kind": "oracle",
            "sample": f"{n_envs} of the {N_ENVS} grids x {EPISODE} steps ({reps} rep), FP64 table + C step, "
                      f"{dt:.1f} s"}


def _oracle_shard(payload):
    """One worker of the env-parallel oracle timing (a spawned process): the
    FP64 table and C rollout of its own grids; returns its wall time."""
    import torch
    torch.set_num_threads(1)
    from oracle import discrete, prob
    cls, dem, ws, wd, F0, drops, params, p_continue, env_ids = payload
    t0 = time.perf_counter()
    q = [prob.table_f32(cls[i][None], dem[i][None], ws[i:i + 1], wd[i:i + 1], params, 30.0)[0].reshape(-1, 8)
         for i in range(len(env_ids))]
    n = len(env_ids)
    ro = discrete.Rollout(np.full(n, SIDE), np.full(n, SIDE), F0.reshape(-1), np.concatenate(q), p_continue,
                          seed=1000, env_ids=np.asarray(env_ids, np.int32))
    ro.step(EPISODE, np.ascontiguousarray(drops))
    return time.perf_counter() - t0


def cpu_parallel(scn, drops, per_core=CPU_SAMPLE_ENVS // 4):
    """The oracle env-parallel: one spawned process per host core, each on its
    own grids of the batch; rate = all grids' cell-updates / the slowest
    worker's time (process start-up excluded)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    n = min(cores * per_core, N_ENVS)
    p = scn.params.as_dict()
    jobs = []
    for w in range(cores):
        env_ids = list(range(w * per_core, min((w + 1) * per_core, n)))
        if not env_ids:
            break
        e0, e1 = env_ids[0], env_ids[-1] + 1
        jobs.append((np.stack([scn.env(e, scn.cls) for e in env_ids]), np.stack([scn.env(e, scn.dem) for e in env_ids]),
                     scn.wind_speed[e0:e1], scn.wind_dir[e0:e1], np.stack([scn.env(e, scn.F0) for e in env_ids]),
                     drops[:, e0:e1], p, scn.params.p_continue, env_ids))
    from concurrent.futures import ProcessPoolExecutor
    try:
        with ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn")) as ex:
            times = list(ex.map(_oracle_shard, jobs))
    except Exception as exc:        # a worker that could not start: report, do not fail the bench
        return {"unavailable": f"env-parallel oracle failed: {type(exc).__name__}: {exc}"[:200]}
    dt = max(times)
    return {"value": n * SIDE * SIDE * EPISODE / dt, "unit": "cell-updates/s", "cores": len(jobs),
            "kind": "oracle",
            "sample": f"{n} of the {N_ENVS} grids x {EPISODE} steps, {per_core} grids per process, "
                      f"slowest process {dt:.1f} s"}


def cpu_relaxed(n=8):
    """The FP64 relaxed oracle (PyTorch CPU, one thread): rates of Eqs. 1-4
    from the parameters under autograd, T = 100 relaxed steps (Eqs. 5-10),
    backward to every parameter; fwd+bwd cell-steps/s."""
    import torch

    from oracle import prob
    from oracle import relaxed as orx
    from paper_2512_06102_gb300 import scenarios
    torch.set_num_threads(1)
    scn = scenarios.make_scenario(SIDE, SIDE, N=n, seed=2)
    f64 = torch.float64
    p = scn.params
    th = [torch.tensor(float(x), dtype=f64, requires_grad=True)
          for x in (p.p_base, p.alpha_w1, p.alpha_w2, p.alpha_s, p.alpha_gamma, p.p_continue)]
    mv = torch.tensor(np.asarray(p.mu_veg, np.float64), requires_grad=True)
    md = torch.tensor(np.asarray(p.mu_den, np.float64), requires_grad=True)
    cls = torch.as_tensor(scn.cls).long().reshape(n, SIDE, SIDE)
    dem = torch.as_tensor(scn.dem).double().reshape(n, SIDE, SIDE)
    F0 = torch.as_tensor(scn.F0).reshape(n, SIDE, SIDE)
    t0 = time.perf_counter()
    r = prob.rates(cls, dem, torch.as_tensor(scn.wind_speed).double(), torch.as_tensor(scn.wind_dir).double(),
                   th[0], th[1], th[2], th[3], th[4], mv, md, p.cell_size)
    ou, ob = orx.relaxed_rollout((F0 <= 1).double(), (F0 == 2).double(), r, th[5], REL_T)
    (0.5 * ou.sum() + ob.sum()).backward()
    dt = time.perf_counter() - t0
    return {"value": n * SIDE * SIDE * REL_T / dt, "unit": "fwd+bwd cell-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} grids of {SIDE}x{SIDE}, T = {REL_T}, FP64 autograd, {dt:.1f} s"}


def cpu_large(side=1024, steps=50):
    """The oracle on one large grid (the dense C sweep costs the same per cell
    at any size, so a {side}^2 grid of the same generator stands for the
    4096^2 ones): FP64 table + 50 steps with drops."""
    import torch

    from oracle import discrete, prob
    from paper_2512_06102_gb300 import scenarios
    torch.set_num_threads(1)
    scn = scenarios.make_scenario(side, side, N=1, seed=0)
    dr = scenarios.drops(steps, scn.H, scn.W, seed=0)
    t0 = time.perf_counter()
    q32 = prob.table_f32(scn.env(0, scn.cls)[None], scn.env(0, scn.dem)[None], scn.wind_speed[:1],
                         scn.wind_dir[:1], scn.params.as_dict(), scn.params.cell_size)[0]
    ro = discrete.Rollout(scn.H, scn.W, scn.F0, q32.reshape(-1, 8), scn.params.p_continue, seed=1000)
    ro.step(steps, np.ascontiguousarray(dr))
    dt = time.perf_counter() - t0
    return {"value": side * side * steps / dt, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"1 grid of {side}x{side} x {steps} steps with drops (FP64 table + C step), {dt:.1f} s"}


def run_reference(args):
    """The reference arm: the oracle as it stands (FP64 table + the plain C
    step), env-parallel over the host cores (one spawned process per core,
    REF_PER_CORE grids each per step), on grids of the benchmark's workload;
    one process if the pool cannot start."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    from paper_2512_06102_gb300 import scenarios
    cores = os.cpu_count() or 1
    n = cores * REF_PER_CORE
    scn = scenarios.make_scenario(SIDE, SIDE, N=n, seed=0)
    drops = scenarios.drops(EPISODE, scn.H, scn.W, seed=0)
    p = scn.params.as_dict()
    jobs = []
    for w in range(cores):
        e0, e1 = w * REF_PER_CORE, (w + 1) * REF_PER_CORE
        ids = list(range(e0, e1))
        jobs.append((np.stack([scn.env(e, scn.cls) for e in ids]), np.stack([scn.env(e, scn.dem) for e in ids]),
                     scn.wind_speed[e0:e1], scn.wind_dir[e0:e1], np.stack([scn.env(e, scn.F0) for e in ids]),
                     drops[:, e0:e1], p, scn.params.p_continue, ids))

    def run_steps(step_fn):
        for _ in range(max(1, args.warmup)):
            step_fn()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step_fn()
        return time.perf_counter() - t0

    used = cores
    try:
        with ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
            dt = run_steps(lambda: list(ex.map(_oracle_shard, jobs)))
    except Exception:           # no process pool: one process on one core
        import torch
        torch.set_num_threads(1)
        used = 1
        dt = run_steps(lambda: [_oracle_shard(j) for j in jobs])
    value = args.steps * n * SIDE * SIDE * EPISODE / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded fBm landcover/DEM stand-ins for WorldCover/GLO-30)",
            "config": {"workload": f"batched: {N_ENVS} grids x {SIDE}x{SIDE}, {EPISODE}-step episode, 3x3 drop/step",
                       "global_batch": N_ENVS * world, "grid": [SIDE, SIDE], "steps_per_episode": EPISODE,
                       "parallelism": f"{used} host processes (env-parallel oracle)"},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": used, "kind": "oracle",
                             "sample": f"each step: {n} of the {N_ENVS} grids x {EPISODE} steps, "
                                       f"{REF_PER_CORE} grids per process"},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile(case: str):
    """Small cases of the workloads for ncu captures (inputs still larger than
    L2, a few GB on the device at most): 'resident' = 1024 grids of 128^2, one
    200-step episode with drops on the fused resident kernel; 'relaxed' = 256
    grids of 128^2, one tiled relaxed forward step, one two-step forward pass,
    two one-step adjoints, sixteen adjoint steps in two-step passes and one 16-step rate-adjoint accumulation; 'tiled' = 2 grids of 4096^2, 800 steps with
    drops on the fused tiled kernel (256 threads a tile, 16 steps a round); 'plain' = the batched
    workload (4096 grids of 128^2, probability table) for 20 steps of the plain one-launch-per-step path;
    'prob' = the probability table of 1024 grids of 128^2."""
    import torch

    from paper_2512_06102_gb300 import build, jwf, scenarios

    build.build()
    dev = torch.device("cuda", 0)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    if case == "prob":
        # the probability table of 1024 grids of 128^2 (q: 537 MB, larger than L2)
        scn = scenarios.make_scenario(SIDE, SIDE, N=1024, seed=0)
        sim = jwf.Sim(SIDE, SIDE, n_envs=1024, n_classes=scenarios.N_CLASSES, seed=0)
        sim.set_params(scn.params)
        sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
        torch.cuda.synchronize()
        print(f"profile case prob: mean q {float(sim.probs()[0].mean()):.6f}")
    elif case == "plain":
        # the plain one-launch-per-step comparator on the batched workload (table path)
        scn = scenarios.make_scenario(SIDE, SIDE, N=N_ENVS, seed=0)
        drops = scenarios.drops(20, scn.H, scn.W, seed=0)
        sim = jwf.Sim(SIDE, SIDE, n_envs=N_ENVS, n_classes=scenarios.N_CLASSES, seed=0)
        sim.set_params(scn.params)
        sim.set_kernel(jwf.KERNEL_PLAIN)
        sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
        sim.load_state(to(scn.F0))
        out = sim.step(20, to(drops))
        torch.cuda.synchronize()
        print(f"profile case plain: burned after 20 steps {int(out[1][-1].sum())}")
    elif case in ("resident", "tiled"):
        N, S, K = (1024, SIDE, EPISODE) if case == "resident" else (2, BIG_SIDE, 800)
        scn = scenarios.make_scenario(S, S, N=N, seed=0)
        drops = scenarios.drops(K, scn.H, scn.W, seed=0)
        sim = jwf.Sim(S, S, n_envs=N, n_classes=scenarios.N_CLASSES, seed=0)
        sim.set_params(scn.params)
        sim.set_terrain(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
        if case == "resident":
            sim.set_kernel(jwf.KERNEL_FUSED)
            sim.set_reorder_steps(0)        # the whole episode in one launch
        else:
            sim.set_kernel(jwf.KERNEL_TILED_FUSED, 256)
            sim.set_round_steps(16)
        sim.load_state(to(scn.F0))
        out = sim.step(K, to(drops))
        torch.cuda.synchronize()
        print(f"profile case {case}: burned at the end {int(out[1][-1].sum())}")
    else:
        scn = scenarios.make_scenario(SIDE, SIDE, N=REL_ENVS, seed=100)
        sim = jwf.Sim(SIDE, SIDE, n_envs=REL_ENVS, n_classes=scenarios.N_CLASSES, keep_rates=True)
        sim.set_params(scn.params)
        sim.precompute_probs(to(scn.cls), to(scn.dem), to(scn.wind_speed), to(scn.wind_dir))
        pb0 = (to(scn.F0) == 2).float()
        pu0 = 1.0 - pb0
        g = torch.Generator(device=dev).manual_seed(3)
        au = torch.randn(pu0.shape, device=dev, generator=g)
        ab = torch.randn(pu0.shape, device=dev, generator=g)
        glam = torch.empty((16, sim.cells), device=dev)
        gpc = torch.zeros(1, dtype=torch.float64, device=dev)
        ou, ob = sim.relaxed_fwd(pu0, pb0)
        two = (torch.empty((2, sim.cells), device=dev), torch.empty((2, sim.cells), device=dev))
        sim.relaxed_fwd_steps(pu0, pb0, two[0], two[1])
        for t in range(2):
            sim.relaxed_bwd(pu0, pb0, au, ab, None, None, None, glam[t], gpc)
        # sixteen adjoint steps in two-step passes (the rollout's backward)
        gu16, gb16 = torch.empty_like(pu0), torch.empty_like(pu0)
        sim.relaxed_bwd_steps(torch.stack([pu0] * 16), torch.stack([pb0] * 16), au, ab, gu16, gb16, glam=glam,
                              gpc=gpc)
        gr = torch.zeros((sim.cells, 8), device=dev)
        sim.rates_accumulate(glam, torch.stack([pb0] * 16), gr)
        torch.cuda.synchronize()
        print(f"profile case relaxed: {float(ou.sum()):.3f} {float(gr.abs().sum()):.3f}")


def main():
    args = parse()
    if args.profile is not None:
        run_profile(args.profile)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
