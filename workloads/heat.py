"""Seeded synthetic inputs shaped like the paper's heat-equation workloads.

The paper's experiments (Sec. 5) use closed-form data on the unit square; the
benchmark workloads here keep the same shapes (m interior points per side with
m + 1 a power of two, N a power of two, T = 1) and replace the data by seeded
random fields:

* ``u0``   -- a smooth random sine series, sum of c_j sin(j pi x) (1D) or
              c_{jl} sin(j pi x) sin(l pi y) (2D), coefficients U[-1, 1];
* ``fsrc`` -- the source f^n at every interior node and step, i.i.d. U[-1, 1];
* ``eps``  -- the epsilon of the block epsilon-circulant preconditioner.

Layouts: a space-time field is ``[N][ny][nx]`` (x fastest), the same order as
u = (u^1; u^2; ...; u^N) in Sec. 2.  Nothing here evaluates the method.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class HeatCase:
    """One all-at-once heat problem: geometry, eps and the seeded data."""

    name: str
    dim: int            # 1 or 2 spatial dimensions
    m: int              # interior points per side, h = 1/(m+1)
    N: int              # number of backward-Euler steps, tau = T/N
    T: float
    eps: float
    u0: np.ndarray      # (m,) or (m, m) = [ny][nx]
    fsrc: np.ndarray    # (N, m) or (N, m, m)
    a: float = 1.0      # constant diffusion coefficient
    seed: int = 0

    @property
    def tau(self) -> float:
        return self.T / self.N

    @property
    def J(self) -> int:
        return self.m ** self.dim

    @property
    def U(self) -> int:
        """Number of space-time unknowns N*J."""
        return self.N * self.J


def grid_points(m: int) -> np.ndarray:
    """Interior nodes x_i = i h, i = 1..m, h = 1/(m+1)."""
    return np.arange(1, m + 1, dtype=np.float64) / (m + 1)


def eps_sqrt_tau(N: int, T: float = 1.0, factor: float = 1.0) -> float:
    return factor * math.sqrt(T / N)


def _sine_series_1d(c: np.ndarray, m: int) -> np.ndarray:
    x = grid_points(m)
    j = np.arange(1, c.size + 1, dtype=np.float64)
    return np.sin(np.pi * np.outer(x, j)) @ c


def _sine_series_2d(c: np.ndarray, m: int) -> np.ndarray:
    """u0[iy, ix] = sum_{jy, jx} c[jy, jx] sin(jx pi x) sin(jy pi y)."""
    x = grid_points(m)
    j = np.arange(1, c.shape[0] + 1, dtype=np.float64)
    s = np.sin(np.pi * np.outer(x, j))          # s[i, j] = sin(j pi x_i)
    return s @ c @ s.T                          # [iy, ix] = s[iy, jy] c[jy, jx] s[ix, jx]


def heat_case_1d(seed: int = 1, m: int = 63, N: int = 64, T: float = 1.0,
                 eps: float | None = None, nterms: int = 8) -> HeatCase:
    """1D heat on (0,1): draws c (nterms) then f (N, m) from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1.0, 1.0, nterms)
    u0 = _sine_series_1d(c, m)
    fsrc = rng.uniform(-1.0, 1.0, (N, m))
    if eps is None:
        eps = eps_sqrt_tau(N, T, 0.5)
    return HeatCase(f"heat1d_m{m}_N{N}", 1, m, N, T, float(eps), u0, fsrc, 1.0, seed)


def heat_case_2d(seed: int = 2, m: int = 255, N: int = 256, T: float = 1.0,
                 eps: float | None = None, nterms: int = 8,
                 dtype=np.float64) -> HeatCase:
    """2D heat on the unit square: draws c (nterms, nterms) then f (N, m, m)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1.0, 1.0, (nterms, nterms))
    u0 = _sine_series_2d(c, m)
    fsrc = rng.uniform(-1.0, 1.0, (N, m, m)).astype(dtype, copy=False)
    if eps is None:
        eps = eps_sqrt_tau(N, T)
    return HeatCase(f"heat2d_m{m}_N{N}", 2, m, N, T, float(eps), u0, fsrc, 1.0, seed)


def batch_cases(seed: int = 4, count: int = 64, sides=(63, 127, 255),
                steps=(32, 64, 128, 256, 512), T: float = 1.0,
                nterms: int = 8) -> list[HeatCase]:
    """Uneven batch: per instance draw side, N, ln eps ~ U[ln 1e-4, ln sqrt(tau)],
    then the sine coefficients and the source, all from one default_rng(seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(rng.choice(sides))
        N = int(rng.choice(steps))
        lo, hi = math.log(1e-4), math.log(math.sqrt(T / N))
        eps = math.exp(rng.uniform(lo, hi))
        c = rng.uniform(-1.0, 1.0, (nterms, nterms))
        u0 = _sine_series_2d(c, m)
        fsrc = rng.uniform(-1.0, 1.0, (N, m, m))
        out.append(HeatCase(f"batch{i}_m{m}_N{N}", 2, m, N, T, eps, u0, fsrc, 1.0, seed))
    return out


def grf_log_coefficient(seed: int = 5, m: int = 255, ell: float = 0.1,
                        sigma: float = 1.0) -> np.ndarray:
    """Gaussian random field g on all (m+2)^2 nodes (boundary included), with the
    squared-exponential covariance sigma^2 exp(-r^2 / (2 ell^2)).  The kernel is
    separable, so g = sigma * A Z A^T with A A^T the 1D kernel matrix
    (A = Q diag(sqrt(max(d, 0))) from its eigendecomposition) and Z ~ N(0, 1).
    Returns g[iy, ix]; the diffusion coefficient is a = exp(g)."""
    rng = np.random.default_rng(seed)
    x = np.arange(m + 2, dtype=np.float64) / (m + 1)
    C = np.exp(-np.subtract.outer(x, x) ** 2 / (2.0 * ell * ell))
    d, Q = np.linalg.eigh(C)
    A = Q * np.sqrt(np.maximum(d, 0.0))
    Z = rng.standard_normal((m + 2, m + 2))
    return sigma * (A @ Z @ A.T)


def circulating_wind_case(m: int = 255, N: int = 256, T: float = 1.0):
    """The data of Example 3 of Sec. 5 on the nodes of (-1, 1)^2 with m
    interior points per side (h = 2/(m+1)): the circulating wind
    w = (2y(1 - x^2), -2x(1 - y^2)) as [2][m+2][m+2] node values ([iy][ix]),
    the hot-wall boundary data g(x, y, t_n) = (1 - exp(-10 t_n)) phi(x, y)
    with phi = 1 on the wall x = 1 and 0 elsewhere, as [N][m+2][m+2] (interior
    entries zero), u0 = 0 and no source.  Returns (wind, g, u0, fsrc)."""
    s = -1.0 + 2.0 * np.arange(m + 2, dtype=np.float64) / (m + 1)
    X, Y = np.meshgrid(s, s)              # X[iy, ix] = x_ix, Y[iy, ix] = y_iy
    wind = np.stack([2.0 * Y * (1.0 - X * X), -2.0 * X * (1.0 - Y * Y)])
    phi = np.zeros((m + 2, m + 2))
    phi[:, m + 1] = 1.0                   # the wall x = 1
    t = T * np.arange(1, N + 1) / N
    g = (1.0 - np.exp(-10.0 * t))[:, None, None] * phi[None, :, :]
    return wind, g, np.zeros((m, m)), np.zeros((N, m, m))
