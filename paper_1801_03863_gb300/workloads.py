"""Seeded synthetic inputs for MinxEnt-LBM runs.

This module is the only code shared by the CUDA path's tests and the oracle's:
it produces macroscopic initial fields (density, velocity) and run parameters,
and holds none of the method's arithmetic (no equilibrium, no collision, no
streaming).  Every array is float64, row-major [y][x] with x fastest.

The setups follow the paper's workloads (Table II: shock tube, lid-driven
cavities) plus a Taylor-Green vortex for the viscosity check.  The paper uses
no external dataset, so nothing here stands in for one.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# --------------------------------------------------------------------------
# Single-instance setups.
# --------------------------------------------------------------------------
def shock_tube_1d(n: int = 800, split: int | None = None, rho_left: float = 1.0,
                  rho_right: float = 0.5):
    """Density step at rest: nodes [0, split) at rho_left, the rest at rho_right.

    Sec. IV.G / Table II row ST (1D form): split defaults to n // 2.
    Returns (rho [1, n], u [1, n]).
    """
    split = n // 2 if split is None else split
    rho = np.full((1, n), rho_right, dtype=np.float64)
    rho[0, :split] = rho_left
    return rho, np.zeros((1, n))


def shock_tube_2d(nx: int = 800, ny: int = 4, rho_left: float = 1.0, rho_right: float = 0.5):
    """The paper's shock tube: D2Q9 (800, 4), constant in y (Table II row ST).

    Returns (rho, ux, uy), each [ny, nx].
    """
    rho = np.full((ny, nx), rho_right, dtype=np.float64)
    rho[:, : nx // 2] = rho_left
    z = np.zeros((ny, nx))
    return rho, z, z.copy()


def taylor_green(n: int, u0: float = 0.02, rho0: float = 1.0, ny: int | None = None):
    """Periodic Taylor-Green vortex on an n x ny lattice (k = 2 pi / n).

    u_x = -u0 cos(kx) sin(ky), u_y = u0 sin(kx) cos(ky), and the
    pressure-consistent density rho0 - (3 rho0 u0^2 / 4)(cos 2kx + cos 2ky)
    (p = rho / 3).  Returns (rho, ux, uy), each [ny, n].
    """
    ny = n if ny is None else ny
    kx = 2.0 * math.pi / n
    ky = 2.0 * math.pi / ny
    x = np.arange(n, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    ux = -u0 * np.cos(kx * x) * np.sin(ky * y)
    uy = u0 * np.sin(kx * x) * np.cos(ky * y)
    rho = rho0 - 0.75 * rho0 * u0 * u0 * (np.cos(2 * kx * x) + np.cos(2 * ky * y))
    return rho, ux, uy


def taylor_green_energy_rate(nu: float, n: int, ny: int | None = None) -> float:
    """Decay rate of the kinetic energy of the vortex above: 2 nu (kx^2 + ky^2)."""
    ny = n if ny is None else ny
    kx = 2.0 * math.pi / n
    ky = 2.0 * math.pi / ny
    return 2.0 * nu * (kx * kx + ky * ky)


def cavity(side: int, rho0: float = 1.0, noise: float = 0.0, seed: int = 0):
    """Lid-driven cavity at rest: rho = rho0 + U(-noise, noise), u = 0.

    Returns (rho, ux, uy), each [side, side].
    """
    rng = np.random.default_rng(seed)
    rho = np.full((side, side), rho0, dtype=np.float64)
    if noise:
        rho += rng.uniform(-noise, noise, size=(side, side))
    z = np.zeros((side, side))
    return rho, z, z.copy()


def nu_from_reynolds(re: float, u_lid: float, side: int) -> float:
    """Kinematic viscosity for Re = U L / nu with L the side in nodes."""
    return u_lid * side / re


# --------------------------------------------------------------------------
# Ensembles.
# --------------------------------------------------------------------------
@dataclass
class CavityMember:
    side: int
    re: float
    u_lid: float
    nu: float


def cavity_ensemble(count: int = 64, seed: int = 0, side_unit: int = 64, side_max_units: int = 16,
                    re_range=(100.0, 1.0e4), u_range=(0.05, 0.1)):
    """Cavities of uneven size and viscosity.

    Per member, in this order: side = side_unit * U{1..side_max_units},
    Re log-uniform in re_range, lid speed uniform in u_range; nu = U side / Re.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        side = side_unit * int(rng.integers(1, side_max_units + 1))
        re = math.exp(rng.uniform(math.log(re_range[0]), math.log(re_range[1])))
        u = float(rng.uniform(u_range[0], u_range[1]))
        out.append(CavityMember(side, re, u, nu_from_reynolds(re, u, side)))
    return out


@dataclass
class TubeMember:
    n: int
    ratio: float
    nu: float


def tube_ensemble(count: int = 4096, seed: int = 1, n_range=(200, 20000),
                  ratio_range=(1.5, 4.0), nu_range=(1e-5, 1e-2)):
    """Shock tubes of uneven length: per member, in this order, N log-uniform
    in n_range (rounded), left/right density ratio uniform, nu log-uniform."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        ratio = float(rng.uniform(*ratio_range))
        nu = math.exp(rng.uniform(math.log(nu_range[0]), math.log(nu_range[1])))
        out.append(TubeMember(n, ratio, nu))
    return out


def tube_fields(member: TubeMember):
    """rho_R = 1, rho_L = ratio, left part = nodes below N // 2, at rest."""
    return shock_tube_1d(member.n, member.n // 2, rho_left=member.ratio, rho_right=1.0)


# --------------------------------------------------------------------------
# Random population states (one-step tests).
# --------------------------------------------------------------------------
# Magnitude profile of a resting D2Q9 / D1Q3 population vector (rest, axis,
# diagonal).  Used only to draw plausible positive states.
_PROFILE9 = np.array([16, 4, 4, 4, 4, 1, 1, 1, 1], dtype=np.float64) / 36.0
_PROFILE3 = np.array([4, 1, 1], dtype=np.float64) / 6.0


def random_populations(q: int, ny: int, nx: int, eps: float = 0.3, rho_spread: float = 0.2,
                       seed: int = 0) -> np.ndarray:
    """Positive random populations [q, ny, nx]: rho(x) * profile * (1 + eps xi),
    rho uniform in [1 - rho_spread, 1 + rho_spread], xi uniform in [-1, 1]."""
    rng = np.random.default_rng(seed)
    prof = _PROFILE9 if q == 9 else _PROFILE3
    rho = rng.uniform(1.0 - rho_spread, 1.0 + rho_spread, size=(ny, nx))
    xi = rng.uniform(-1.0, 1.0, size=(q, ny, nx))
    return rho[None] * prof[:, None, None] * (1.0 + eps * xi)
