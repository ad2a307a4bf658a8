"""ctypes binding of libjwf (include/jwf.h): argument marshalling only.

Every computation runs in libjwf's CUDA kernels; this module turns torch
tensors into device pointers and the current torch stream into the
cudaStream_t argument.  There is no CPU fallback: loading fails loudly when
libjwf has not been built.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libjwf.so")

JWF_AUTO_RESET = 0x1
JWF_WIND_PER_CELL = 0x2
JWF_KEEP_RATES = 0x4

KERNEL_AUTO, KERNEL_PLAIN, KERNEL_RESIDENT, KERNEL_FUSED, KERNEL_TILED, KERNEL_TILED_FUSED = 0, 1, 2, 3, 4, 5
RELAXED_TILED, RELAXED_PLAIN = 0, 1

STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error",
          4: "device wait timed out", 5: "call out of order", 6: "unsupported"}


class JwfError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class _Config(ctypes.Structure):
    _fields_ = [("n_envs", ctypes.c_int32), ("h_H", ctypes.POINTER(ctypes.c_int32)),
                ("h_W", ctypes.POINTER(ctypes.c_int32)), ("n_classes", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("t_max", ctypes.c_int32), ("drop_radius", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


class _Params(ctypes.Structure):
    _fields_ = [("p_base", ctypes.c_float), ("alpha_w1", ctypes.c_float), ("alpha_w2", ctypes.c_float),
                ("alpha_s", ctypes.c_float), ("alpha_gamma", ctypes.c_float), ("p_continue", ctypes.c_float),
                ("cell_size", ctypes.c_float), ("h_mu_veg", ctypes.POINTER(ctypes.c_float)),
                ("h_mu_den", ctypes.POINTER(ctypes.c_float))]


# exported symbol -> (restype, argtypes)
_VP = ctypes.c_void_p
_SIGS = {
    "jwf_create": (ctypes.c_int, [ctypes.POINTER(_Config), ctypes.POINTER(_VP)]),
    "jwf_destroy": (ctypes.c_int, [_VP]),
    "jwf_set_params": (ctypes.c_int, [_VP, ctypes.POINTER(_Params)]),
    "jwf_sync": (ctypes.c_int, [_VP, _VP]),
    "jwf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "jwf_last_error": (ctypes.c_char_p, [_VP]),
    "jwf_n_envs": (ctypes.c_int32, [_VP]),
    "jwf_n_cells": (ctypes.c_int64, [_VP]),
    "jwf_env_offset": (ctypes.c_int64, [_VP, ctypes.c_int32]),
    "jwf_precompute_probs": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "jwf_set_probs": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "jwf_set_terrain": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "jwf_get_probs": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    "jwf_check_prob_bound": (ctypes.c_int, [_VP, ctypes.c_int64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "jwf_load_state": (ctypes.c_int, [_VP, _VP, _VP]),
    "jwf_reset": (ctypes.c_int, [_VP, _VP, _VP]),
    "jwf_apply_action": (ctypes.c_int, [_VP, _VP, _VP]),
    "jwf_step": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP]),
    "jwf_set_kernel": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int32]),
    "jwf_set_relaxed_kernel": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "jwf_set_wind_series": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP]),
    "jwf_step_record": (ctypes.c_int, [_VP, ctypes.c_int32] + [_VP] * 6),
    "jwf_set_seed": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "jwf_packed_size": (ctypes.c_int64, [ctypes.c_int64]),
    "jwf_pack_states": (ctypes.c_int, [ctypes.c_int64, _VP, _VP, _VP]),
    "jwf_unpack_states": (ctypes.c_int, [ctypes.c_int64, _VP, _VP, _VP]),
    "jwf_load_state_packed": (ctypes.c_int, [_VP, _VP, _VP]),
    "jwf_get_state_packed": (ctypes.c_int, [_VP, _VP, _VP]),
    "jwf_step_record_packed": (ctypes.c_int, [_VP, ctypes.c_int32] + [_VP] * 6),
    "jwf_agent_reset": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP, _VP]),
    "jwf_agent_step": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, _VP, _VP,
                                      ctypes.c_int32, _VP, _VP]),
    "jwf_state_planes": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP]),
    "jwf_set_pair_counter": (ctypes.c_int, [_VP, _VP]),
    "jwf_size_classes": (ctypes.c_int32, [_VP, _VP]),
    "jwf_set_class_threads": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32]),
    "jwf_set_round_steps": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "jwf_set_env_priority": (ctypes.c_int, [_VP, _VP]),
    "jwf_set_tile_copy": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "jwf_set_reorder_steps": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "jwf_tile_copy": (ctypes.c_int32, [_VP]),
    "jwf_set_tile_copy_wait": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_int32]),
    "jwf_get_state": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    "jwf_step_relaxed_fwd": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "jwf_step_relaxed_bwd": (ctypes.c_int, [_VP] * 11),
    "jwf_rates_bwd": (ctypes.c_int, [_VP, ctypes.c_int32] + [_VP] * 9),
    "jwf_rates_accumulate": (ctypes.c_int, [_VP, ctypes.c_int32] + [_VP] * 5),
    "jwf_relaxed_fwd_steps": (ctypes.c_int, [_VP, ctypes.c_int32] + [_VP] * 6),
    "jwf_relaxed_bwd_steps": (ctypes.c_int, [_VP, ctypes.c_int32] + [_VP] * 10),
    "jwf_rates_contract": (ctypes.c_int, [_VP] * 8),
    "jwf_mask_words": (ctypes.c_int64, [ctypes.c_int64]),
    "jwf_pack_masks": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _VP, _VP, _VP]),
    "jwf_step_masked": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP]),
    "jwf_step_relaxed_bwd_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP,
                                                    ctypes.c_float] + [_VP] * 9),
}
NOALLOC_MAX_CELLS = 1 << 22
EXPORTS = tuple(_SIGS)

_lib = None


def lib() -> ctypes.CDLL:
    """Load libjwf (built by paper_2512_06102_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libjwf is not built ({LIB_PATH} missing): run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_cuda:
            raise ValueError("libjwf takes device tensors")
        if not t.is_contiguous():
            raise ValueError("libjwf takes contiguous tensors")
        return t.data_ptr()
    return int(t)


def packed_size(n_cells: int) -> int:
    """Bytes of a 2-bit packed row of n states (ceil(n / 4) rounded up to 16)."""
    return int(lib().jwf_packed_size(int(n_cells)))


def pack_states(states: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """uint8 states (device, any shape, n elements) -> 2-bit packed uint8
    [packed_size(n)] (cell i in bits 2(i mod 4).. of byte i // 4)."""
    n = states.numel()
    if out is None:
        out = torch.zeros(packed_size(n), dtype=torch.uint8, device=states.device)
    st = lib().jwf_pack_states(n, _ptr(states), _ptr(out), _stream(stream))
    if st != 0:
        raise RuntimeError(f"jwf_pack_states: {lib().jwf_status_string(st).decode()}")
    return out


def unpack_states(packed: torch.Tensor, n_cells: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """2-bit packed states -> uint8 [n_cells]."""
    if out is None:
        out = torch.empty(int(n_cells), dtype=torch.uint8, device=packed.device)
    st = lib().jwf_unpack_states(int(n_cells), _ptr(packed), _ptr(out), _stream(stream))
    if st != 0:
        raise RuntimeError(f"jwf_unpack_states: {lib().jwf_status_string(st).decode()}")
    return out


def mask_words(n_cells: int) -> int:
    """uint32 words of one bit-packed action mask row of n cells."""
    return int(lib().jwf_mask_words(int(n_cells)))


def pack_masks(masks: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """uint8 action masks [k, cells] (device, nonzero = water) -> bit rows
    int32 [k, mask_words(cells)] (cell g at bit g % 32 of word g // 32)."""
    if masks.dim() != 2 or masks.dtype != torch.uint8:
        raise ValueError("masks must be uint8 [k, cells]")
    k, n = masks.shape
    if out is None:
        out = torch.empty((k, mask_words(n)), dtype=torch.int32, device=masks.device)
    st = lib().jwf_pack_masks(int(k), int(n), _ptr(masks.contiguous()), _ptr(out), _stream(stream))
    if st != 0:
        raise RuntimeError(f"jwf_pack_masks: {lib().jwf_status_string(st).decode()}")
    return out


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class _DevView:
    """Zero-copy torch view of a device pointer owned by libjwf."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                          "data": (int(ptr), False), "version": 3, "strides": None}


def _view(ptr: int, shape, dtype: torch.dtype) -> torch.Tensor:
    typestr = {torch.uint8: "|u1", torch.int32: "<i4", torch.float32: "<f4"}[dtype]
    return torch.as_tensor(_DevView(ptr, shape, typestr), device="cuda")


@dataclass
class ParamSet:
    p_base: float = 0.58
    alpha_w1: float = 0.045
    alpha_w2: float = 0.131
    alpha_s: float = 0.078
    alpha_gamma: float = 1.0
    p_continue: float = 0.5
    cell_size: float = 30.0
    mu_veg: np.ndarray | None = None
    mu_den: np.ndarray | None = None

    @staticmethod
    def from_any(p) -> "ParamSet":
        if isinstance(p, ParamSet):
            return p
        d = p if isinstance(p, dict) else p.__dict__
        keys = ParamSet.__dataclass_fields__.keys()
        return ParamSet(**{k: d[k] for k in keys if k in d})


def relaxed_bwd_noalloc(n_envs: int, H: int, W: int, r, p_continue: float, pun, pburn, gun_out, gburn_out,
                        mask=None, gun=None, gburn=None, gpc=None, stream=None):
    """jwf_step_relaxed_bwd_noalloc: the relaxed adjoint step for a uniform
    batch without a context, for callers that cannot allocate device memory
    (the library allocates nothing; output tensors the caller does not pass
    are created here, by torch).  Returns (gun, gburn)."""
    cells = int(n_envs) * int(H) * int(W)
    if int(n_envs) < 1 or int(H) < 1 or int(W) < 1:
        raise ValueError("n_envs, H and W must be positive")
    if gun is None:
        gun = torch.empty_like(pun)
    if gburn is None:
        gburn = torch.empty_like(pburn)
    # the library takes raw pointers: check every buffer against the sizes
    # the call implies before it can read or write past an end
    planes = {"pun": pun, "pburn": pburn, "gun_out": gun_out, "gburn_out": gburn_out, "gun": gun,
              "gburn": gburn, "mask": mask}
    device = r.device if isinstance(r, torch.Tensor) else None
    for name, t, n, dt in ([("r", r, 8 * cells, torch.float32)]
                           + [(k, v, cells, torch.float32) for k, v in planes.items()]
                           + [("gpc", gpc, 1, torch.float64)]):
        if t is None:
            continue
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if t.numel() != n:
            raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
        if t.device != device:
            raise ValueError(f"{name} is on {t.device}, r on {device}")
    st = lib().jwf_step_relaxed_bwd_noalloc(int(n_envs), int(H), int(W), _ptr(r), ctypes.c_float(p_continue),
                                            _ptr(pun), _ptr(pburn), _ptr(mask), _ptr(gun_out), _ptr(gburn_out),
                                            _ptr(gun), _ptr(gburn), _ptr(gpc), _stream(stream))
    if st != 0:
        raise JwfError(st, "jwf_step_relaxed_bwd_noalloc")
    return gun, gburn


class Sim:
    """A batch of wildfire grids on the current CUDA device (one jwf_ctx)."""

    def __init__(self, H, W, n_envs: int | None = None, n_classes: int = 11, seed: int = 0,
                 t_max: int = 0, drop_radius: int = 1, auto_reset: bool = False,
                 wind_per_cell: bool = False, keep_rates: bool = False):
        L = lib()
        if np.isscalar(H):
            assert n_envs is not None
            Hs = np.full(n_envs, int(H), np.int32)
            Ws = np.full(n_envs, int(W), np.int32)
        else:
            Hs = np.ascontiguousarray(H, np.int32)
            Ws = np.ascontiguousarray(W, np.int32)
        self.H, self.W = Hs, Ws
        self.N = int(Hs.shape[0])
        self.n_classes = int(n_classes)
        flags = ((JWF_AUTO_RESET if auto_reset else 0) | (JWF_WIND_PER_CELL if wind_per_cell else 0)
                 | (JWF_KEEP_RATES if keep_rates else 0))
        cfg = _Config(self.N, Hs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                      Ws.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), self.n_classes,
                      ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF), int(t_max), int(drop_radius), flags)
        torch.cuda.init()
        h = _VP()
        st = L.jwf_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != 0:
            raise JwfError(st, "jwf_create")
        self._h = h
        self.cells = int(L.jwf_n_cells(h))
        self.offsets = np.array([L.jwf_env_offset(h, e) for e in range(self.N + 1)], np.int64)
        self.params: ParamSet | None = None
        self.tables_version = 0         # bumped by every call that changes the rate tables

    # -- plumbing -----------------------------------------------------------
    def _check(self, st: int, where: str):
        if st != 0:
            raise JwfError(st, where, lib().jwf_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().jwf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self, stream=None):
        self._check(lib().jwf_sync(self._h, _stream(stream)), "jwf_sync")

    # -- parameters and tables ---------------------------------------------
    def set_params(self, p):
        self.tables_version += 1
        p = ParamSet.from_any(p)
        mv = np.ascontiguousarray(p.mu_veg, np.float32)
        md = np.ascontiguousarray(p.mu_den, np.float32)
        assert mv.shape == (self.n_classes,) and md.shape == (self.n_classes,)
        cp = _Params(p.p_base, p.alpha_w1, p.alpha_w2, p.alpha_s, p.alpha_gamma, p.p_continue, p.cell_size,
                     mv.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                     md.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        self._check(lib().jwf_set_params(self._h, ctypes.byref(cp)), "jwf_set_params")
        self.params = p

    def precompute_probs(self, cls, dem, wind_speed, wind_dir, stream=None):
        self.tables_version += 1
        self._terrain = (cls, dem, wind_speed, wind_dir)
        self._check(lib().jwf_precompute_probs(self._h, _ptr(cls), _ptr(dem), _ptr(wind_speed), _ptr(wind_dir),
                                               _stream(stream)), "jwf_precompute_probs")

    def set_terrain(self, cls, dem, wind_speed, wind_dir, stream=None):
        """Register (borrow) the terrain the fused step evaluates probabilities from."""
        self._terrain = (cls, dem, wind_speed, wind_dir)     # keep the buffers alive
        self._check(lib().jwf_set_terrain(self._h, _ptr(cls), _ptr(dem), _ptr(wind_speed), _ptr(wind_dir),
                                          _stream(stream)), "jwf_set_terrain")

    def set_wind_series(self, wind_speed=None, wind_dir=None, stream=None):
        """Per-step wind, float [steps, N] each (None: back to static wind)."""
        if wind_speed is None:
            self._wser = None
            self._check(lib().jwf_set_wind_series(self._h, 0, None, None, _stream(stream)), "jwf_set_wind_series")
            return
        self._wser = (wind_speed, wind_dir)     # keep the borrowed buffers alive
        self._check(lib().jwf_set_wind_series(self._h, int(wind_speed.shape[0]), _ptr(wind_speed), _ptr(wind_dir),
                                              _stream(stream)), "jwf_set_wind_series")

    def set_probs(self, q, r=None, stream=None):
        self.tables_version += 1
        self._check(lib().jwf_set_probs(self._h, _ptr(q), _ptr(r), _stream(stream)), "jwf_set_probs")

    def probs(self):
        """Borrowed views (q, r) of the context's tables, float32 [cells, 8]."""
        q, r = _VP(), _VP()
        self._check(lib().jwf_get_probs(self._h, ctypes.byref(q), ctypes.byref(r)), "jwf_get_probs")
        qt = _view(q.value, (self.cells, 8), torch.float32)
        rt = _view(r.value, (self.cells, 8), torch.float32) if r.value else None
        return qt, rt

    def check_prob_bound(self, class_v, class_u, z_v, z_u, wexp, direction, stream=None):
        """jwf_check_prob_bound: (p_f, B, p) float32 [n, 3] of the fused step's
        two-level ignition probability for n pair tuples (wexp float32 [n, 2]
        as hi, lo)."""
        n = int(class_v.numel())
        for name, t, k, dt in (("class_v", class_v, n, torch.uint8), ("class_u", class_u, n, torch.uint8),
                               ("z_v", z_v, n, torch.float32), ("z_u", z_u, n, torch.float32),
                               ("wexp", wexp, 2 * n, torch.float32), ("direction", direction, n, torch.int32)):
            if not isinstance(t, torch.Tensor) or t.dtype != dt or t.numel() != k:
                raise ValueError(f"{name} must be a {dt} tensor of {k} elements")
        out = torch.empty((n, 3), dtype=torch.float32, device=class_v.device)
        self._check(lib().jwf_check_prob_bound(self._h, n, _ptr(class_v), _ptr(class_u), _ptr(z_v), _ptr(z_u),
                                               _ptr(wexp), _ptr(direction), _ptr(out), _stream(stream)),
                    "jwf_check_prob_bound")
        return out

    # -- discrete simulation -----------------------------------------------
    def load_state(self, F0, stream=None):
        self._check(lib().jwf_load_state(self._h, _ptr(F0), _stream(stream)), "jwf_load_state")

    def load_state_packed(self, P0, stream=None):
        """Initial states as 2-bit packed bytes (pack_states of uint8 [cells])."""
        self._check(lib().jwf_load_state_packed(self._h, _ptr(P0), _stream(stream)), "jwf_load_state_packed")

    def state_packed(self, out=None, stream=None) -> torch.Tensor:
        """The current state, 2-bit packed: uint8 [packed_size(cells)]."""
        if out is None:
            out = torch.zeros(packed_size(self.cells), dtype=torch.uint8,
                              device=torch.device("cuda", torch.cuda.current_device()))
        self._check(lib().jwf_get_state_packed(self._h, _ptr(out), _stream(stream)), "jwf_get_state_packed")
        return out

    def reset(self, env_mask=None, stream=None):
        self._check(lib().jwf_reset(self._h, _ptr(env_mask), _stream(stream)), "jwf_reset")

    def apply_action(self, mask, stream=None):
        self._check(lib().jwf_apply_action(self._h, _ptr(mask), _stream(stream)), "jwf_apply_action")

    def set_kernel(self, kernel: int = KERNEL_AUTO, threads_per_env: int = 0):
        self._check(lib().jwf_set_kernel(self._h, int(kernel), int(threads_per_env)), "jwf_set_kernel")

    def set_relaxed_kernel(self, kernel: int = RELAXED_TILED):
        self._check(lib().jwf_set_relaxed_kernel(self._h, int(kernel)), "jwf_set_relaxed_kernel")

    def size_classes(self) -> list:
        buf = (ctypes.c_int32 * 4)()
        n = lib().jwf_size_classes(self._h, ctypes.cast(buf, _VP))
        return [int(buf[i]) for i in range(n)]

    def set_class_threads(self, size_class: int, threads: int):
        self._check(lib().jwf_set_class_threads(self._h, int(size_class), int(threads)), "jwf_set_class_threads")

    def set_round_steps(self, steps: int):
        self._check(lib().jwf_set_round_steps(self._h, int(steps)), "jwf_set_round_steps")

    def set_reorder_steps(self, steps: int = 32):
        """Resident kernels: after `steps` steps, restart the launch with the
        envs with the most burning cells first (0: one launch)."""
        self._check(lib().jwf_set_reorder_steps(self._h, int(steps)), "jwf_set_reorder_steps")

    def set_tile_copy(self, tma: bool = True):
        """Tiled kernels: stage regions with TMA tensor copies (True) or loads."""
        self._check(lib().jwf_set_tile_copy(self._h, int(bool(tma))), "jwf_set_tile_copy")

    def set_tile_copy_wait(self, timeout_ns: int = 2_000_000_000, no_copy: bool = False):
        """Bound of the tiled kernels' tensor-copy wait; no_copy (diagnostics)
        arms the wait without a copy so that it runs out."""
        self._check(lib().jwf_set_tile_copy_wait(self._h, ctypes.c_uint64(int(timeout_ns)), int(bool(no_copy))),
                    "jwf_set_tile_copy_wait")

    def tile_copy(self) -> bool:
        return bool(lib().jwf_tile_copy(self._h))

    def set_env_priority(self, priority=None):
        """Resident-kernel scheduling hint: envs with a higher priority (host
        float [N], e.g. expected fire duration) are started first; None
        restores the default order."""
        if priority is None:
            self._check(lib().jwf_set_env_priority(self._h, None), "jwf_set_env_priority")
            return
        pr = np.ascontiguousarray(np.asarray(priority, np.float32).reshape(-1))
        if pr.size != self.N:
            raise ValueError("priority must have one value per env")
        self._check(lib().jwf_set_env_priority(self._h, pr.ctypes.data), "jwf_set_env_priority")

    def set_pair_counter(self, counter):
        """counter: int64 device tensor of four elements (pairs compared,
        candidate Philox blocks, remain-burning draws, words scanned), or None."""
        self._check(lib().jwf_set_pair_counter(self._h, _ptr(counter)), "jwf_set_pair_counter")

    def step_masked(self, k: int, mask_bits, burning=None, burnt=None, done=None, stream=None):
        """Advance k steps with each step's action as a bit-packed cell mask
        (pack_masks): int32 [k, mask_words(cells)].  Returns (burning, burnt,
        done) [k, N]."""
        if (mask_bits.dtype != torch.int32 or mask_bits.dim() != 2
                or tuple(mask_bits.shape) != (k, mask_words(self.cells))):
            raise ValueError("mask_bits must be int32 [k, mask_words(cells)]")
        dev = torch.device("cuda", torch.cuda.current_device())
        if burning is None:
            burning = torch.empty((k, self.N), dtype=torch.int32, device=dev)
        if burnt is None:
            burnt = torch.empty((k, self.N), dtype=torch.int32, device=dev)
        if done is None:
            done = torch.empty((k, self.N), dtype=torch.uint8, device=dev)
        self._check(lib().jwf_step_masked(self._h, int(k), _ptr(mask_bits), _ptr(burning), _ptr(burnt), _ptr(done),
                                          _stream(stream)), "jwf_step_masked")
        return burning, burnt, done

    def step(self, k: int = 1, drops=None, burning=None, burnt=None, done=None, stream=None, history=None,
             packed: bool = False):
        """Advance k steps; returns the (burning, burnt, done) tensors [k, N].
        history: optional uint8 [k, cells] device tensor that receives the
        state after every step (jwf_step_record), or with packed=True uint8
        [k, packed_size(cells)] that receives it 2-bit packed
        (jwf_step_record_packed)."""
        dev = torch.device("cuda", torch.cuda.current_device())
        if burning is None:
            burning = torch.empty((k, self.N), dtype=torch.int32, device=dev)
        if burnt is None:
            burnt = torch.empty((k, self.N), dtype=torch.int32, device=dev)
        if done is None:
            done = torch.empty((k, self.N), dtype=torch.uint8, device=dev)
        if history is None:
            self._check(lib().jwf_step(self._h, int(k), _ptr(drops), _ptr(burning), _ptr(burnt), _ptr(done),
                                       _stream(stream)), "jwf_step")
        elif packed:
            if tuple(history.shape) != (k, packed_size(self.cells)) or history.dtype != torch.uint8:
                raise ValueError("packed history must be uint8 [k, packed_size(cells)]")
            self._check(lib().jwf_step_record_packed(self._h, int(k), _ptr(drops), _ptr(burning), _ptr(burnt),
                                                     _ptr(done), _ptr(history), _stream(stream)),
                        "jwf_step_record_packed")
        else:
            if tuple(history.shape) != (k, self.cells) or history.dtype != torch.uint8:
                raise ValueError("history must be uint8 [k, cells]")
            self._check(lib().jwf_step_record(self._h, int(k), _ptr(drops), _ptr(burning), _ptr(burnt), _ptr(done),
                                              _ptr(history), _stream(stream)), "jwf_step_record")
        return burning, burnt, done

    def agent_reset(self, agent, water0: int, random_fire: bool = True, obs_k: int = 5, obs=None, stream=None):
        self._check(lib().jwf_agent_reset(self._h, _ptr(agent), int(water0), int(bool(random_fire)), int(obs_k),
                                          _ptr(obs), _stream(stream)), "jwf_agent_reset")

    def agent_step(self, actions, agent, water0: int, random_fire: bool = True, burn_penalty: float = 0.01,
                   reward=None, done=None, obs_k: int = 5, obs=None, stream=None):
        self._check(lib().jwf_agent_step(self._h, _ptr(actions), _ptr(agent), int(water0), int(bool(random_fire)),
                                         ctypes.c_float(burn_penalty), _ptr(reward), _ptr(done), int(obs_k),
                                         _ptr(obs), _stream(stream)), "jwf_agent_step")

    def set_seed(self, seed: int):
        self._check(lib().jwf_set_seed(self._h, ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF)), "jwf_set_seed")

    def state_planes(self, states, pun=None, pburn=None, stream=None):
        """uint8 [n, cells] states -> float (p_un, p_burn) planes [n, cells]."""
        if pun is None:
            pun = torch.empty(states.shape, dtype=torch.float32, device=states.device)
        if pburn is None:
            pburn = torch.empty(states.shape, dtype=torch.float32, device=states.device)
        n = states.shape[0] if states.dim() == 2 else 1
        self._check(lib().jwf_state_planes(self._h, int(n), _ptr(states), _ptr(pun), _ptr(pburn), _stream(stream)),
                    "jwf_state_planes")
        return pun, pburn

    def state_views(self):
        """Borrowed views (state uint8 [cells], t int32 [N], episode int32 [N])."""
        s, t, e = _VP(), _VP(), _VP()
        self._check(lib().jwf_get_state(self._h, ctypes.byref(s), ctypes.byref(t), ctypes.byref(e)),
                    "jwf_get_state")
        return (_view(s.value, (self.cells,), torch.uint8), _view(t.value, (self.N,), torch.int32),
                _view(e.value, (self.N,), torch.int32))

    def state(self) -> torch.Tensor:
        return self.state_views()[0].clone()

    # -- relaxed update ----------------------------------------------------
    def relaxed_fwd(self, pun, pburn, mask=None, pun_out=None, pburn_out=None, stream=None):
        if pun_out is None:
            pun_out = torch.empty_like(pun)
        if pburn_out is None:
            pburn_out = torch.empty_like(pburn)
        self._check(lib().jwf_step_relaxed_fwd(self._h, _ptr(pun), _ptr(pburn), _ptr(mask), _ptr(pun_out),
                                               _ptr(pburn_out), _stream(stream)), "jwf_step_relaxed_fwd")
        return pun_out, pburn_out

    def relaxed_bwd(self, pun, pburn, gun_out, gburn_out, mask=None, gun=None, gburn=None, glam=None,
                    gpc=None, stream=None):
        if gun is None:
            gun = torch.empty_like(pun)
        if gburn is None:
            gburn = torch.empty_like(pburn)
        self._check(lib().jwf_step_relaxed_bwd(self._h, _ptr(pun), _ptr(pburn), _ptr(mask), _ptr(gun_out),
                                               _ptr(gburn_out), _ptr(gun), _ptr(gburn), _ptr(glam), _ptr(gpc),
                                               _stream(stream)), "jwf_step_relaxed_bwd")
        return gun, gburn

    def relaxed_fwd_steps(self, pun, pburn, pun_out, pburn_out, masks=None, stream=None):
        """pun_out / pburn_out [n, cells]: row t = state after step t."""
        n = pun_out.shape[0]
        self._check(lib().jwf_relaxed_fwd_steps(self._h, int(n), _ptr(pun), _ptr(pburn), _ptr(masks),
                                                _ptr(pun_out), _ptr(pburn_out), _stream(stream)),
                    "jwf_relaxed_fwd_steps")
        return pun_out, pburn_out

    def relaxed_bwd_steps(self, pun, pburn, gun_out, gburn_out, gun, gburn, masks=None, glam=None, gpc=None,
                          stream=None):
        """pun / pburn [n, cells]: row t = state before step t; adjoints of
        the state after step n-1 in, of the state before step 0 out."""
        n = pun.shape[0]
        self._check(lib().jwf_relaxed_bwd_steps(self._h, int(n), _ptr(pun), _ptr(pburn), _ptr(masks),
                                                _ptr(gun_out), _ptr(gburn_out), _ptr(gun), _ptr(gburn),
                                                _ptr(glam), _ptr(gpc), _stream(stream)), "jwf_relaxed_bwd_steps")
        return gun, gburn

    def rates_bwd(self, glam, pburn, cls, dem, wind_speed, wind_dir, gparams, mask=None, stream=None):
        n = glam.shape[0] if glam.dim() == 2 else 1
        self._check(lib().jwf_rates_bwd(self._h, int(n), _ptr(glam), _ptr(pburn), _ptr(mask), _ptr(cls),
                                        _ptr(dem), _ptr(wind_speed), _ptr(wind_dir), _ptr(gparams),
                                        _stream(stream)), "jwf_rates_bwd")
        return gparams

    def rates_accumulate(self, glam, pburn, gr, mask=None, stream=None):
        n = glam.shape[0] if glam.dim() == 2 else 1
        self._check(lib().jwf_rates_accumulate(self._h, int(n), _ptr(glam), _ptr(pburn), _ptr(mask), _ptr(gr),
                                               _stream(stream)), "jwf_rates_accumulate")
        return gr

    def rates_contract(self, gr, cls, dem, wind_speed, wind_dir, gparams, stream=None):
        self._check(lib().jwf_rates_contract(self._h, _ptr(gr), _ptr(cls), _ptr(dem), _ptr(wind_speed),
                                             _ptr(wind_dir), _ptr(gparams), _stream(stream)), "jwf_rates_contract")
        return gparams

    @property
    def grad_size(self) -> int:
        return 5 + 2 * self.n_classes
