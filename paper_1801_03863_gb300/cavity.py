"""Lid-driven cavity studies of Sec. IV.H-I, run through the library.

* LDSS (Sec. IV.H, Table II): many 17 x 17 cavities at rest with rho = 2.7,
  one per (1/tau, lid speed) pair, advanced 1000 steps in one batched
  context.  A run is stable when every population stays finite and
  non-negative at every node and step; the library's per-instance
  ``unstable`` counter (status word A11) records exactly that criterion, so
  the sweep needs no host-side inspection of the fields.
* LDAS (Sec. IV.I): a 257 x 257 cavity at Re = 1000, run to a steady stream
  function; the stream function comes from ``lbm_stream_function`` (device
  Simpson/trapezoid integration of u_y), the vortex centres are its extrema,
  normalised by the lid speed as in the paper.

The helpers here only organise runs and read off extrema; every time step
and the stream-function integration run in the library's kernels.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import lbm, workloads as wl

LDSS_SIDE = 17
LDSS_RHO = 2.7
LDSS_STEPS = 1000
LDAS_SIDE = 257
LDAS_RHO = 2.7


def nu_from_inv_tau(inv_tau: float) -> float:
    """Eq. (visco-tau): nu = (tau - 1/2) / 3."""
    return (1.0 / inv_tau - 0.5) / 3.0


@dataclasses.dataclass
class StabilityMap:
    inv_tau: np.ndarray          # [T]
    u_lid: np.ndarray            # [U], increasing
    stable: np.ndarray           # [T, U] bool
    unstable_nodes: np.ndarray   # [T, U] counter value (node-steps)

    def max_stable_lid(self) -> np.ndarray:
        """Largest lid speed of each 1/tau below which every run is stable
        (the paper lowers the lid speed until the run survives); 0 if none."""
        out = np.zeros(len(self.inv_tau))
        for i in range(len(self.inv_tau)):
            ok = self.stable[i]
            k = 0
            while k < len(ok) and ok[k]:
                k += 1
            out[i] = self.u_lid[k - 1] if k > 0 else 0.0
        return out


def ldss_sweep(inv_tau, u_lid, collision: str = "minxent4", compute: str = "f64",
               storage: str | None = None, steps: int = LDSS_STEPS,
               side: int = LDSS_SIDE, rho0: float = LDSS_RHO,
               tau2_reading: str = "printed") -> StabilityMap:
    """One batched context of len(inv_tau) x len(u_lid) cavities (row-major
    over (1/tau, u_lid)), `steps` steps, per-instance stability verdicts."""
    inv_tau = np.asarray(inv_tau, dtype=np.float64)
    u_lid = np.asarray(u_lid, dtype=np.float64)
    pairs = [(t, u) for t in inv_tau for u in u_lid]
    dims = [(side, side)] * len(pairs)
    nus = [nu_from_inv_tau(t) for t, _ in pairs]
    uls = [u for _, u in pairs]
    rho = np.full(side * side * len(pairs), rho0)
    z = np.zeros_like(rho)
    with lbm.Lattice("d2q9", dims, nus, "cavity", u_lid=uls, compute=compute, storage=storage,
                     collision=collision, rho0=rho0, tau2_reading=tau2_reading) as lat:
        lat.init(rho, z, z)
        lat.step(steps)
        counts = np.array([lat.status_instance(i)["unstable"] for i in range(len(pairs))])
    counts = counts.reshape(len(inv_tau), len(u_lid))
    return StabilityMap(inv_tau, u_lid, counts == 0, counts)


# ----------------------------------------------------------------------------
# LDAS: stream function and vortex centres.
# ----------------------------------------------------------------------------
def normalised_stream_function(psi: np.ndarray, u_lid: float) -> np.ndarray:
    """psi in lattice units (node spacing 1) -> psi / (|u_lid| L), L = n - 1
    node spacings between the wall nodes."""
    return psi / (abs(u_lid) * (psi.shape[1] - 1))


def vortex_centres(psi_hat: np.ndarray) -> dict:
    """Extrema of the normalised stream function (the vortex centres of
    Table IV): the main vortex is the minimum over the whole cavity, the
    lower-right and lower-left secondary vortices the maxima over the lower
    right and lower left quadrants.  Positions x_hat = i / (n - 1) (and
    likewise y) from the bottom-left wall node."""
    ny, nx = psi_hat.shape
    out = {}
    j, i = np.unravel_index(np.argmin(psi_hat), psi_hat.shape)
    out["main"] = (float(psi_hat[j, i]), i / (nx - 1), j / (ny - 1), int(i), int(j))
    half_x, half_y = nx // 2, ny // 2
    for name, xs in (("lower_right", slice(half_x, nx)), ("lower_left", slice(0, half_x))):
        q = psi_hat[:half_y, xs]
        jj, ii = np.unravel_index(np.argmax(q), q.shape)
        ii += xs.start
        out[name] = (float(psi_hat[jj, ii]), ii / (nx - 1), jj / (ny - 1), int(ii), int(jj))
    return out


def ldas_cavity(side: int = LDAS_SIDE, re: float = 1000.0, u_lid: float = 0.01,
                collision: str = "minxent4", compute: str = "f64", storage: str | None = None,
                tol: float = 1e-5, check_every: int = 20_000, max_steps: int = 3_000_000,
                rho0: float = LDAS_RHO):
    """Run the LDAS cavity (at rest, rho = rho0, nu = u_lid side / Re) until
    the normalised stream-function minimum changes by less than `tol`
    between checks (Table II's stopping condition).  Table II allows lid
    speeds 0.01 or 0.1; at 0.1 (lattice Mach number 0.17) the compressibility
    error weakens the vortices by a few per cent, at 0.01 the run needs
    ~1.4 M steps at Re = 1000.  Returns (psi_hat, rho, ux, uy, steps)."""
    nu = wl.nu_from_reynolds(re, u_lid, side)
    rho = np.full((side, side), rho0)
    z = np.zeros_like(rho)
    with lbm.Lattice("d2q9", [(side, side)], nu, "cavity", u_lid=u_lid, compute=compute,
                     storage=storage, collision=collision, rho0=rho0) as lat:
        lat.init(rho, z, z)
        prev, steps = None, 0
        while steps < max_steps:
            lat.step(check_every)
            steps += check_every
            psi_hat = normalised_stream_function(lat.stream_function().reshape(side, side), u_lid)
            cur = float(psi_hat.min())
            if prev is not None and abs(cur - prev) < tol:
                break
            prev = cur
        r, x, y = lat.moments()
    return psi_hat, r.reshape(side, side), x.reshape(side, side), y.reshape(side, side), steps


def ldas_batch(u_lids, side: int = LDAS_SIDE, re: float = 1000.0, collision: str = "minxent4",
               compute: str = "f64", storage: str | None = None, tol: float = 1e-5,
               check_every: int = 20_000, max_steps: int = 3_000_000, rho0: float = LDAS_RHO):
    """Several LDAS cavities (one per lid speed, same side and Re) advanced
    together in one batched context, each checked with its own stream
    function (``lbm_stream_function_batch``: one member read back, not the
    whole ensemble) until every member meets Table II's stopping rule.
    Returns a list of (psi_hat, steps at which the member converged)."""
    u_lids = [float(u) for u in u_lids]
    n = len(u_lids)
    nus = [wl.nu_from_reynolds(re, u, side) for u in u_lids]
    rho = np.full(side * side * n, rho0)
    z = np.zeros_like(rho)
    prev = [None] * n
    done = [None] * n
    psi = [None] * n
    with lbm.Lattice("d2q9", [(side, side)] * n, nus, "cavity", u_lid=u_lids, compute=compute,
                     storage=storage, collision=collision, rho0=rho0) as lat:
        lat.init(rho, z, z)
        steps = 0
        while steps < max_steps and any(d is None for d in done):
            lat.step(check_every)
            steps += check_every
            for i, u in enumerate(u_lids):
                if done[i] is not None:
                    continue
                psi[i] = normalised_stream_function(lat.stream_function_instance(i), u)
                cur = float(psi[i].min())
                if prev[i] is not None and abs(cur - prev[i]) < tol:
                    done[i] = steps
                prev[i] = cur
    return [(psi[i], done[i] if done[i] is not None else steps) for i in range(n)]
