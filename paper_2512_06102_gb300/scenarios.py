"""Seeded synthetic scenarios shaped like the JaxWildfire workloads.

This module only draws inputs (landcover classes, elevation, wind, initial
fires, tanker drops) and holds default parameter values; it contains none of
the fire model's arithmetic.  The same arrays feed the CUDA path and the CPU
oracle.

The paper builds its maps from ESA WorldCover landcover and the Copernicus
GLO-30 DEM (arXiv 2512.06102, Section 3 "Data integrations"); neither is
available offline, so seeded fractal fields stand in for them at the same
30 m cell size:
  * landcover: 11 WorldCover-like classes obtained by thresholding one fBm field
    at the cumulative class fractions below (about 10% non-burnable);
  * DEM: an independent fBm field min-max scaled to [0, 2000] m;
  * wind: per grid, speed U(0, 10) m/s and direction U(0, 2 pi);
  * fires: 1-3 distinct burnable cells per grid;
  * tanker: one drop centre per grid per step, uniform over the grid (a 3x3
    drop, clipped at the edges, is expanded by the step itself).
fBm = 6 octaves of bilinear value noise, persistence 0.5, lacunarity 2; the
coarsest lattice spacing is 1/4 of the grid side (at least 1 cell).
Every grid e draws from numpy.random.default_rng(seed * 1_000_003 + e).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# class id, name, fraction of the map, mu_veg, mu_den  (values are this
# project's choice: the paper prints no class table)
CLASSES = [
    (0, "tree", 0.25, 0.4, 0.3),
    (1, "shrub", 0.15, 0.2, 0.1),
    (2, "grass", 0.20, 0.0, -0.2),
    (3, "crop", 0.15, -0.3, -0.2),
    (4, "wetland", 0.05, -0.5, -0.4),
    (5, "mangrove", 0.03, -0.4, 0.0),
    (6, "moss_lichen", 0.07, -0.6, -0.6),
    (7, "water", 0.05, 0.0, -1.0),
    (8, "built", 0.03, 0.0, -1.0),
    (9, "bare", 0.015, 0.0, -1.0),
    (10, "snow", 0.005, 0.0, -1.0),
]
N_CLASSES = len(CLASSES)
# order of the classes along the landcover field, low to high values
_FIELD_ORDER = [7, 4, 5, 3, 8, 2, 1, 0, 6, 9, 10]

STATE_NOFUEL, STATE_CANBURN, STATE_BURNING, STATE_BURNT = 0, 1, 2, 3


@dataclass
class Params:
    """Model parameters (Eqs. 1-4 and the stochastic update)."""
    p_base: float = 0.58
    alpha_w1: float = 0.045
    alpha_w2: float = 0.131
    alpha_s: float = 0.078          # per degree of slope
    alpha_gamma: float = 1.0
    p_continue: float = 0.5
    cell_size: float = 30.0         # metres
    mu_veg: np.ndarray = field(default_factory=lambda: np.array([c[3] for c in CLASSES], np.float32))
    mu_den: np.ndarray = field(default_factory=lambda: np.array([c[4] for c in CLASSES], np.float32))

    def as_dict(self):
        return dict(p_base=self.p_base, alpha_w1=self.alpha_w1, alpha_w2=self.alpha_w2,
                    alpha_s=self.alpha_s, alpha_gamma=self.alpha_gamma, p_continue=self.p_continue,
                    cell_size=self.cell_size, mu_veg=np.asarray(self.mu_veg, np.float32),
                    mu_den=np.asarray(self.mu_den, np.float32))


def burnable_classes(mu_den) -> np.ndarray:
    """Classes with fuel (mu_den > -1).  Input encoding only."""
    return np.asarray(mu_den) > -1.0


@dataclass
class Scenario:
    H: np.ndarray            # int32 [N]
    W: np.ndarray            # int32 [N]
    cls: np.ndarray          # uint8 [cells] concatenated
    dem: np.ndarray          # float32 [cells]
    wind_speed: np.ndarray   # float32 [N]
    wind_dir: np.ndarray     # float32 [N]
    F0: np.ndarray           # uint8 [cells] initial states
    params: Params

    @property
    def N(self) -> int:
        return int(self.H.shape[0])

    @property
    def offsets(self) -> np.ndarray:
        sizes = self.H.astype(np.int64) * self.W.astype(np.int64)
        return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)

    @property
    def uniform(self) -> bool:
        return bool((self.H == self.H[0]).all() and (self.W == self.W[0]).all())

    def env(self, e: int, a: np.ndarray) -> np.ndarray:
        o = self.offsets
        return a[o[e]:o[e + 1]].reshape(int(self.H[e]), int(self.W[e]), *a.shape[1:])

    def stacked(self, a: np.ndarray) -> np.ndarray:
        """[N, H, W, ...] view of a concatenated array (uniform batches only)."""
        assert self.uniform
        return a.reshape(self.N, int(self.H[0]), int(self.W[0]), *a.shape[1:])


def _octave_spacings(H: int, W: int, octaves: int = 6):
    sp, out = max(1.0, min(H, W) / 4.0), []
    for _ in range(octaves):
        out.append(sp)
        sp = max(1.0, sp / 2.0)
    return out


def _lattice_shape(H: int, W: int, spacing: float):
    return int(math.ceil(H / spacing)) + 2, int(math.ceil(W / spacing)) + 2


def _device():
    import torch
    return torch.device("cuda") if torch.cuda.is_available() else torch.device("cpu")


def _interp(lat, H: int, W: int, spacing: float):
    """Bilinear value noise for a batch of lattices [n, gh, gw] -> [n, H, W]
    (separable: along x on the lattice rows, then along y).  float64 torch."""
    import torch
    dev = lat.device
    ys = torch.arange(H, dtype=torch.float64, device=dev) / spacing
    xs = torch.arange(W, dtype=torch.float64, device=dev) / spacing
    y0 = torch.floor(ys).long()
    x0 = torch.floor(xs).long()
    fy = (ys - y0)[None, :, None]
    fx = (xs - x0)[None, None, :]
    rows = lat.index_select(2, x0) * (1 - fx) + lat.index_select(2, x0 + 1) * fx     # [n, gh, W]
    return rows.index_select(1, y0) * (1 - fy) + rows.index_select(1, y0 + 1) * fy


def _fbm_batch(lats, H: int, W: int):
    """fBm from per-octave lattices (list over octaves of [n, gh, gw] numpy)."""
    import torch
    dev = _device()
    amp, norm = 1.0, 0.0
    total = None
    for lat, sp in zip(lats, _octave_spacings(H, W)):
        v = amp * _interp(torch.as_tensor(lat, device=dev), H, W, sp)
        total = v if total is None else total + v
        norm += amp
        amp *= 0.5
    return total / norm


def _landcover_batch(field_):
    """Threshold each grid's field at its own cumulative class quantiles
    (linear-interpolated order statistics, numpy's default definition)."""
    import torch
    n = field_.shape[0]
    flat = field_.reshape(n, -1)
    srt, _ = torch.sort(flat, dim=1)
    m = flat.shape[1]
    fr = np.array([CLASSES[c][2] for c in _FIELD_ORDER])
    qs = np.cumsum(fr)[:-1] / fr.sum()
    idx = torch.zeros(flat.shape, dtype=torch.long, device=flat.device)
    for q in qs:
        pos = q * (m - 1)
        lo = int(math.floor(pos))
        hi = min(lo + 1, m - 1)
        cut = srt[:, lo] + (srt[:, hi] - srt[:, lo]) * (pos - lo)
        idx += (flat >= cut[:, None]).long()
    order = torch.as_tensor(np.asarray(_FIELD_ORDER, np.uint8), device=flat.device)
    return order[idx].reshape(field_.shape)


def _draw_env(seed: int, e: int, H: int, W: int, n_ign=(1, 3)):
    """All random draws of grid e, in a fixed order, from its own stream."""
    rng = np.random.default_rng(seed * 1_000_003 + e)
    sps = _octave_spacings(H, W)
    lat_c = [rng.random(_lattice_shape(H, W, sp)) for sp in sps]
    lat_z = [rng.random(_lattice_shape(H, W, sp)) for sp in sps]
    V = rng.uniform(0.0, 10.0)
    Th = rng.uniform(0.0, 2.0 * math.pi)
    k = int(rng.integers(n_ign[0], n_ign[1] + 1))
    pick_u = rng.random(n_ign[1])          # positions among the burnable cells
    return lat_c, lat_z, V, Th, k, pick_u


def _make_group(seed: int, envs, H: int, W: int, chunk: int = 1024):
    """Grids `envs` (all H x W): cls, dem, V, Th, F0 arrays in env order."""
    burn_cls = burnable_classes(np.array([c[4] for c in CLASSES]))
    out = []
    for c0 in range(0, len(envs), chunk):
        ids = envs[c0:c0 + chunk]
        draws = [_draw_env(seed, e, H, W) for e in ids]
        nO = len(draws[0][0])
        cls = _landcover_batch(_fbm_batch([np.stack([d[0][o] for d in draws]) for o in range(nO)], H, W))
        cls = cls.cpu().numpy()
        z = _fbm_batch([np.stack([d[1][o] for d in draws]) for o in range(nO)], H, W)
        zmin = z.reshape(len(ids), -1).amin(dim=1)[:, None, None]
        zmax = z.reshape(len(ids), -1).amax(dim=1)[:, None, None]
        z = ((z - zmin) / (zmax - zmin).clamp_min(1e-12) * 2000.0).cpu().numpy()
        burn = burn_cls[cls]
        F = np.where(burn, STATE_CANBURN, STATE_NOFUEL).astype(np.uint8)
        for i, d in enumerate(draws):
            cand = np.flatnonzero(burn[i].reshape(-1))
            if cand.size:
                # distinct cells: sample without replacement by successive picks
                chosen = []
                pool = cand.copy()
                for j in range(min(d[4], cand.size)):
                    t = int(d[5][j] * pool.size)
                    chosen.append(pool[t])
                    pool = np.delete(pool, t)
                F[i].reshape(-1)[chosen] = STATE_BURNING
        for i, d in enumerate(draws):
            out.append((cls[i].reshape(-1), z[i].astype(np.float32).reshape(-1), np.float32(d[2]),
                        np.float32(d[3]), F[i].reshape(-1)))
    return out


def make_scenario(H, W, N: int | None = None, seed: int = 0, params: Params | None = None) -> Scenario:
    """Batch of N grids; H, W ints (uniform batch) or int sequences (ragged)."""
    if np.isscalar(H):
        assert N is not None
        Hs = np.full(N, int(H), np.int32)
        Ws = np.full(N, int(W), np.int32)
    else:
        Hs = np.asarray(H, np.int32)
        Ws = np.asarray(W, np.int32)
    n = len(Hs)
    parts = [None] * n
    shapes = {}
    for e in range(n):
        shapes.setdefault((int(Hs[e]), int(Ws[e])), []).append(e)
    for (h, w), envs in shapes.items():
        for e, part in zip(envs, _make_group(seed, envs, h, w)):
            parts[e] = part
    return Scenario(H=Hs, W=Ws,
                    cls=np.concatenate([p[0] for p in parts]),
                    dem=np.concatenate([p[1] for p in parts]),
                    wind_speed=np.array([p[2] for p in parts], np.float32),
                    wind_dir=np.array([p[3] for p in parts], np.float32),
                    F0=np.concatenate([p[4] for p in parts]),
                    params=params or Params())


def plain_single_env(H: int = 64, W: int = 64) -> Scenario:
    """One grid of one burnable class (mu_veg = mu_den = 0), flat, no wind,
    one ignition at the centre cell (the single-environment workload)."""
    p = Params(mu_veg=np.zeros(1, np.float32), mu_den=np.zeros(1, np.float32))
    F = np.full(H * W, STATE_CANBURN, np.uint8)
    F[(H // 2) * W + W // 2] = STATE_BURNING
    return Scenario(H=np.array([H], np.int32), W=np.array([W], np.int32),
                    cls=np.zeros(H * W, np.uint8), dem=np.zeros(H * W, np.float32),
                    wind_speed=np.zeros(1, np.float32), wind_dir=np.zeros(1, np.float32),
                    F0=F, params=p)


def ragged_sides(n: int, lo: int = 32, hi: int = 512, seed: int = 0) -> np.ndarray:
    """Square grid sides drawn log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed * 1_000_003 + 999_999_937)
    s = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))
    return np.clip(np.round(s), lo, hi).astype(np.int32)


def drops(k: int, H, W, seed: int = 0, p_drop: float = 1.0) -> np.ndarray:
    """Tanker drop centres int32 [k, N, 2] = (column, row); (-1, -1) = no drop."""
    Hs = np.asarray(H, np.int64).reshape(-1)
    Ws = np.asarray(W, np.int64).reshape(-1)
    rng = np.random.default_rng(seed * 1_000_003 + 424_242_421)
    n = Hs.shape[0]
    x = np.floor(rng.random((k, n)) * Ws[None, :]).astype(np.int32)
    y = np.floor(rng.random((k, n)) * Hs[None, :]).astype(np.int32)
    on = rng.random((k, n)) < p_drop
    out = np.stack([np.where(on, x, -1), np.where(on, y, -1)], axis=-1).astype(np.int32)
    return np.ascontiguousarray(out)
