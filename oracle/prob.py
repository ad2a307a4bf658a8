"""FP64 oracle for the per-(cell, direction) ignition rates of JaxWildfire.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.

Written from arXiv 2512.06102, Section 3 ("Directional propagation" and
"Ignition probability"), Eqs. 1-4, in plain PyTorch float64 so that autograd
can differentiate the rates with respect to the parameters.

Conventions (where the paper leaves them open):
  * direction d = 0..7 has angle d*pi/4 (east = 0, counter-clockwise, Eq. 1);
    Delta_d = (dx, dy) with dy positive northward; rows grow southward, so the
    row offset of Delta_d is -dy;
  * the wind direction Theta is the direction the wind blows toward: spread is
    fastest when the propagation angle equals Theta;
  * slope S(u, d) is the terrain angle in degrees from the source u up to the
    neighbour u + Delta_d: atan((z(u+Delta_d) - z(u)) / (L * |Delta_d|));
  * rate r(v, d) = gamma(v) * phi(u, d) with u = v - Delta_d; r = 0 when u lies
    outside the grid; q(v, d) = 1 - exp(-r(v, d)).
"""
from __future__ import annotations

import math

import torch

# column step and row step of Delta_d (rows grow southward)
DX = (1, 1, 0, -1, -1, -1, 0, 1)
DR = (0, -1, -1, -1, 0, 1, 1, 1)


def shift_from_source(a: torch.Tensor, d: int, fill: float = 0.0) -> torch.Tensor:
    """out[..., y, x] = a[..., y - DR[d], x - DX[d]]: the value at the source
    u = v - Delta_d seen from target v; `fill` where u is off the grid."""
    H, W = a.shape[-2], a.shape[-1]
    out = torch.full_like(a, fill)
    sy, sx = DR[d], DX[d]
    # target rows y with 0 <= y - sy < H, columns x with 0 <= x - sx < W
    y0, y1 = max(0, sy), min(H, H + sy)
    x0, x1 = max(0, sx), min(W, W + sx)
    if y1 > y0 and x1 > x0:
        out[..., y0:y1, x0:x1] = a[..., y0 - sy:y1 - sy, x0 - sx:x1 - sx]
    return out


def inside_mask(H: int, W: int, d: int) -> torch.Tensor:
    """1 where the source u = v - Delta_d of target v lies inside the grid."""
    return shift_from_source(torch.ones(H, W, dtype=torch.float64), d, 0.0)


def slope_degrees(dem: torch.Tensor, cell_size: float) -> torch.Tensor:
    """S(u, d) of Eq. 2 for every source cell u and direction d, in degrees.

    dem: [..., H, W] float64 elevations (metres).  Returns [..., H, W, 8];
    entries whose neighbour u + Delta_d is off the grid are 0 (never used)."""
    H, W = dem.shape[-2], dem.shape[-1]
    out = []
    for d in range(8):
        # neighbour value z(u + Delta_d) at u: shift by -Delta_d
        nb = torch.zeros_like(dem)
        sy, sx = -DR[d], -DX[d]
        y0, y1 = max(0, sy), min(H, H + sy)
        x0, x1 = max(0, sx), min(W, W + sx)
        nb[..., y0:y1, x0:x1] = dem[..., y0 - sy:y1 - sy, x0 - sx:x1 - sx]
        dist = cell_size * (math.sqrt(2.0) if d % 2 == 1 else 1.0)
        valid = torch.zeros_like(dem)
        valid[..., y0:y1, x0:x1] = 1.0
        s = torch.rad2deg(torch.atan((nb - dem) / dist)) * valid
        out.append(s)
    return torch.stack(out, dim=-1)


def rates(cls: torch.Tensor, dem: torch.Tensor, wind_speed: torch.Tensor,
          wind_dir: torch.Tensor, p_base, alpha_w1, alpha_w2, alpha_s, alpha_gamma,
          mu_veg: torch.Tensor, mu_den: torch.Tensor, cell_size: float = 30.0) -> torch.Tensor:
    """r(v, d) = gamma(v) * phi(v - Delta_d, d) for one batch of equal-shaped grids.

    cls: int64 [N, H, W] landcover class; dem: float64 [N, H, W];
    wind_speed, wind_dir: float64 [N] (per grid) or [N, H, W] (per cell);
    parameters: python floats or float64 0-d tensors (may require grad);
    mu_veg, mu_den: float64 [C] per-class vegetation / density modifiers.
    Returns float64 [N, H, W, 8], indexed by target v and direction d.
    """
    N, H, W = cls.shape
    f64 = torch.float64
    V = wind_speed.to(f64)
    Th = wind_dir.to(f64)
    if V.dim() == 1:
        V = V.view(N, 1, 1).expand(N, H, W)
        Th = Th.view(N, 1, 1).expand(N, H, W)
    veg = mu_veg[cls]
    den = mu_den[cls]
    S = slope_degrees(dem.to(f64), cell_size)                    # [N,H,W,8] at the source
    # Eq. 3 without the directional factors, at the source u
    base = p_base * (1.0 + veg) * (1.0 + den)                    # [N,H,W]
    # gamma(v) at the target (Section 3, below Eq. 3)
    gamma = alpha_gamma * (1.0 + veg) * (1.0 + den)              # [N,H,W]
    out = []
    for d in range(8):
        ang = d * math.pi / 4.0
        k_wind = torch.exp(alpha_w1 * V) * torch.exp(alpha_w2 * V * (torch.cos(ang - Th) - 1.0))  # Eq. 1
        k_slope = torch.exp(alpha_s * S[..., d])                                                 # Eq. 2
        phi = base * k_wind * k_slope                                                            # Eq. 3
        phi_at_target = shift_from_source(phi, d, 0.0)           # phi(v - Delta_d, d)
        out.append(gamma * phi_at_target)                        # gamma(v) * phi(u, Delta_{u->v})
    return torch.stack(out, dim=-1)


def thresholds(r: torch.Tensor) -> torch.Tensor:
    """q = 1 - exp(-r): per-neighbour ignition probability (Eq. 4 for one burning source)."""
    return -torch.expm1(-r)


def table_f32(cls, dem, wind_speed, wind_dir, params, cell_size: float = 30.0):
    """(q, r) as float32 numpy arrays [N, H, W, 8]: FP64 values rounded to nearest.

    params: dict with p_base, alpha_w1, alpha_w2, alpha_s, alpha_gamma, mu_veg, mu_den."""
    import numpy as np
    t = lambda a: torch.as_tensor(np.asarray(a))
    r = rates(t(cls).long(), t(dem).double(), t(wind_speed).double(), t(wind_dir).double(),
              float(params["p_base"]), float(params["alpha_w1"]), float(params["alpha_w2"]),
              float(params["alpha_s"]), float(params["alpha_gamma"]),
              torch.as_tensor(np.asarray(params["mu_veg"], dtype=np.float64)),
              torch.as_tensor(np.asarray(params["mu_den"], dtype=np.float64)), cell_size)
    q = thresholds(r)
    return q.numpy().astype(np.float32), r.numpy().astype(np.float32), q.numpy(), r.numpy()
