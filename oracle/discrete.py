"""ctypes access to the C oracle (jwf_oracle.c).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
benchmark's CPU-baseline leg.  `build()` compiles the C file with gcc into
oracle/_build/ (plain -O2, no vectorisation flags that change results).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jwf_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_jwf.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile jwf_oracle.c to a shared library; return its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    # -ffp-contract=off: the oracle's float compare must not be fused
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER
            u8p, u32p, i32p, i64p, f32p = (P(ctypes.c_uint8), P(ctypes.c_uint32), P(ctypes.c_int32),
                                           P(ctypes.c_int64), P(ctypes.c_float))
            L.orc_philox4x32_10_batch.argtypes = [ctypes.c_int64, u32p, u32p, u32p]
            L.orc_philox4x32_10_batch.restype = None
            L.orc_uniform24.argtypes = [ctypes.c_uint32]
            L.orc_uniform24.restype = ctypes.c_float
            L.orc_drop_mask.argtypes = [ctypes.c_int] * 5 + [u8p]
            L.orc_drop_mask.restype = None
            L.orc_discrete_step.argtypes = [ctypes.c_int, ctypes.c_int, u8p, u8p, f32p, ctypes.c_float,
                                            u8p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_uint32, i32p, i32p]
            L.orc_discrete_step.restype = None
            L.orc_discrete_rollout.argtypes = [ctypes.c_int, i32p, i32p, i64p, u8p, u8p, f32p,
                                               ctypes.c_float, i32p, ctypes.c_int, ctypes.c_uint64,
                                               i32p, i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               i32p, i32p, u8p, i32p]
            L.orc_discrete_rollout.restype = None
            L.orc_discrete_rollout_masks.argtypes = [ctypes.c_int, i32p, i32p, i64p, u8p, u8p, f32p,
                                                     ctypes.c_float, u8p, ctypes.c_int64, ctypes.c_uint64,
                                                     i32p, i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                     i32p, i32p, u8p, i32p]
            L.orc_discrete_rollout_masks.restype = None
            L.orc_mc_outcomes.argtypes = [ctypes.c_int, ctypes.c_int, u8p, f32p, ctypes.c_float, u8p,
                                          ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_int64, u8p]
            L.orc_mc_outcomes.restype = None
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None, ctype):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox(counters: np.ndarray, key) -> np.ndarray:
    """counters uint32 [n, 4]; key (k0, k1) -> uint32 [n, 4]."""
    c = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros_like(c)
    lib().orc_philox4x32_10_batch(c.shape[0], _ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                                  _ptr(out, ctypes.c_uint32))
    return out


def uniform24(word: int) -> float:
    return float(lib().orc_uniform24(int(word)))


def drop_mask(H: int, W: int, cx: int, cy: int, R: int = 1) -> np.ndarray:
    m = np.zeros((H, W), dtype=np.uint8)
    lib().orc_drop_mask(H, W, cx, cy, R, _ptr(m, ctypes.c_uint8))
    return m


def step(F: np.ndarray, q: np.ndarray, p_continue: float, seed: int = 0, env: int = 0,
         t: int = 0, episode: int = 0, mask: np.ndarray | None = None):
    """One step of one grid.  F uint8 [H, W]; q float32 [H, W, 8]."""
    H, W = F.shape
    Fi = np.ascontiguousarray(F, dtype=np.uint8)
    Fo = np.empty_like(Fi)
    qf = np.ascontiguousarray(q, dtype=np.float32)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    nb = ctypes.c_int32(0)
    nd = ctypes.c_int32(0)
    lib().orc_discrete_step(H, W, _ptr(Fi, ctypes.c_uint8), _ptr(Fo, ctypes.c_uint8),
                            _ptr(qf, ctypes.c_float), ctypes.c_float(p_continue),
                            _ptr(m, ctypes.c_uint8), ctypes.c_uint64(seed), env, t, episode,
                            ctypes.byref(nb), ctypes.byref(nd))
    return Fo, nb.value, nd.value


def mc_outcomes(F: np.ndarray, q: np.ndarray, p_continue: float, n_trials: int, seed: int = 0,
                t: int = 0, episode: int = 0, mask: np.ndarray | None = None) -> np.ndarray:
    """n_trials independent one-step outcomes of grid F -> uint8 [n_trials, H, W]."""
    H, W = F.shape
    Fi = np.ascontiguousarray(F, dtype=np.uint8)
    qf = np.ascontiguousarray(q, dtype=np.float32)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    out = np.empty((n_trials, H, W), np.uint8)
    lib().orc_mc_outcomes(H, W, _ptr(Fi, ctypes.c_uint8), _ptr(qf, ctypes.c_float),
                          ctypes.c_float(p_continue), _ptr(m, ctypes.c_uint8), ctypes.c_uint64(seed),
                          t, episode, n_trials, _ptr(out, ctypes.c_uint8))
    return out


class Rollout:
    """Batch of (possibly ragged) grids advanced by the C oracle.

    H, W: int sequences per env.  F0: concatenated uint8 initial states.
    q: concatenated float32 [cells, 8] table.  drops passed to step() are
    [k, N, 2] for these N grids.  env_ids: the env index of each grid in the
    random-number counter (default 0..N-1)."""

    def __init__(self, H, W, F0: np.ndarray, q: np.ndarray, p_continue: float, seed: int = 0,
                 t_max: int = 0, auto_reset: bool = False, radius: int = 1, env_ids=None):
        self.H = np.ascontiguousarray(H, dtype=np.int32)
        self.W = np.ascontiguousarray(W, dtype=np.int32)
        self.N = int(self.H.shape[0])
        sizes = self.H.astype(np.int64) * self.W.astype(np.int64)
        self.off = np.ascontiguousarray(np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64))
        self.F0 = np.ascontiguousarray(F0, dtype=np.uint8).reshape(-1)
        assert self.F0.size == int(sizes.sum())
        self.F = self.F0.copy()
        self.q = np.ascontiguousarray(q, dtype=np.float32).reshape(-1, 8)
        assert self.q.shape[0] == self.F0.size
        self.p_continue = float(p_continue)
        self.seed = int(seed)
        self.t = np.zeros(self.N, dtype=np.int32)
        self.episode = np.zeros(self.N, dtype=np.int32)
        self.t_max = int(t_max)
        self.auto_reset = bool(auto_reset)
        self.radius = int(radius)
        self.env_ids = None if env_ids is None else np.ascontiguousarray(env_ids, dtype=np.int32)

    def step(self, k: int, drops: np.ndarray | None = None):
        """Advance k steps; drops int32 [k, N, 2] (column, row) or None.
        Returns (burning [k, N], burnt [k, N], done [k, N])."""
        burning = np.zeros((k, self.N), dtype=np.int32)
        burnt = np.zeros((k, self.N), dtype=np.int32)
        done = np.zeros((k, self.N), dtype=np.uint8)
        dr = None if drops is None else np.ascontiguousarray(drops, dtype=np.int32).reshape(k, self.N, 2)
        lib().orc_discrete_rollout(
            self.N, _ptr(self.H, ctypes.c_int32), _ptr(self.W, ctypes.c_int32),
            _ptr(self.off, ctypes.c_int64), _ptr(self.F, ctypes.c_uint8), _ptr(self.F0, ctypes.c_uint8),
            _ptr(self.q, ctypes.c_float), ctypes.c_float(self.p_continue), _ptr(dr, ctypes.c_int32),
            self.radius, ctypes.c_uint64(self.seed), _ptr(self.t, ctypes.c_int32),
            _ptr(self.episode, ctypes.c_int32), k, self.t_max, int(self.auto_reset),
            _ptr(burning, ctypes.c_int32), _ptr(burnt, ctypes.c_int32), _ptr(done, ctypes.c_uint8),
            _ptr(self.env_ids, ctypes.c_int32))
        return burning, burnt, done

    def step_masks(self, masks: np.ndarray):
        """Advance k steps with the tanker action of each step as a cell mask:
        masks uint8 [k, cells] of this batch (nonzero = water).  Returns
        (burning [k, N], burnt [k, N], done [k, N])."""
        m = np.ascontiguousarray(masks, dtype=np.uint8)
        k = int(m.shape[0])
        assert m.size == k * self.F.size
        burning = np.zeros((k, self.N), dtype=np.int32)
        burnt = np.zeros((k, self.N), dtype=np.int32)
        done = np.zeros((k, self.N), dtype=np.uint8)
        lib().orc_discrete_rollout_masks(
            self.N, _ptr(self.H, ctypes.c_int32), _ptr(self.W, ctypes.c_int32),
            _ptr(self.off, ctypes.c_int64), _ptr(self.F, ctypes.c_uint8), _ptr(self.F0, ctypes.c_uint8),
            _ptr(self.q, ctypes.c_float), ctypes.c_float(self.p_continue), _ptr(m, ctypes.c_uint8),
            ctypes.c_int64(self.F.size), ctypes.c_uint64(self.seed), _ptr(self.t, ctypes.c_int32),
            _ptr(self.episode, ctypes.c_int32), k, self.t_max, int(self.auto_reset),
            _ptr(burning, ctypes.c_int32), _ptr(burnt, ctypes.c_int32), _ptr(done, ctypes.c_uint8),
            _ptr(self.env_ids, ctypes.c_int32))
        return burning, burnt, done

    def env_state(self, e: int) -> np.ndarray:
        n = int(self.H[e]) * int(self.W[e])
        return self.F[self.off[e]:self.off[e] + n].reshape(int(self.H[e]), int(self.W[e]))


def pack_states(F: np.ndarray) -> np.ndarray:
    """2-bit packed storage of states 0..3: cell i of the flattened array goes
    to bits 2(i mod 4) and 2(i mod 4) + 1 of byte i // 4 (ceil(n / 4) bytes).
    A storage format of this library, not part of the method."""
    f = np.asarray(F, np.uint8).reshape(-1)
    out = np.zeros((f.size + 3) // 4, np.uint8)
    for j in range(4):
        part = f[j::4].astype(np.uint16) & 3
        out[:part.size] |= (part << (2 * j)).astype(np.uint8)
    return out


def unpack_states(P: np.ndarray, n: int) -> np.ndarray:
    """Inverse of pack_states: the first n states of a packed byte array."""
    p = np.asarray(P, np.uint8).reshape(-1)
    i = np.arange(n)
    return ((p[i // 4] >> (2 * (i % 4))) & 3).astype(np.uint8)
