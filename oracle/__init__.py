"""FP64 CPU oracle for MinxEnt-LBM (Wilson, Pugh & Dawson, arXiv:1801.03863).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow reference the CUDA
path is checked against.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product package never
does, and the two share no code.

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, nested loops); this
module compiles it with gcc on first use and wraps it with ctypes.  Each
wrapped function names the passage of the paper the C function follows.

Pins: every function here is pinned by ``tests/test_oracle_pins.py`` against
facts the paper or the mathematics fix (orthogonality of T, closed-form
equilibrium moments, exact conservation, the u = 0 fixed point, Gibbs'
inequality, an independent Lagrange-dual solution of the constrained
minimisation, D1Q3 = BGK, Taylor-Green decay at the viscosity of
Eq. visco-tau, bounce-back round trips).  No function is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

D1Q3, D2Q9 = 1, 2
BC_PERIODIC, BC_ZERO_GRADIENT, BC_CAVITY = 0, 1, 2
MINXENT4, SRT, MINXENT2, MRT, TRT, NONE = 0, 1, 2, 3, 4, 9
NEWTON_SKIPPED, UNSTABLE = 1, 2
START_HYBRID, START_EQUILIBRIUM = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into ``liblbm_oracle.so``."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
           "-fvisibility=hidden", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        D, I, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        sigs = {
            "orc_d2q9_tables": (None, [P, P, P, P]),
            "orc_d1q3_tables": (None, [P, P]),
            "orc_d2q9_feq": (None, [D, D, D, P]),
            "orc_d1q3_feq": (None, [D, D, P]),
            "orc_kld": (D, [I, P, P]),
            "orc_tau2": (D, [D]),
            "orc_tau_from_nu": (D, [D]),
            "orc_d2q9_minxent": (I, [P, D, D, I, I, P]),
            "orc_d2q9_minxent_converged": (I, [P, D, D, I, D, I, P, P]),
            "orc_d2q9_srt": (I, [P, D, P]),
            "orc_d2q9_mrt": (I, [P, D, D, I, P]),
            "orc_d1q3_minxent": (I, [P, D, P]),
            "orc_d1q3_srt": (I, [P, D, P]),
            "orc_create": (P, [I, I, I, D, I, I, D, D]),
            "orc_destroy": (None, [P]),
            "orc_set_start": (None, [P, I]),
            "orc_set_tau2": (None, [P, D]),
            "orc_init": (None, [P, P, P, P]),
            "orc_set_f": (None, [P, P]),
            "orc_get_f": (None, [P, P]),
            "orc_step": (None, [P, I]),
            "orc_moments": (None, [P, P, P, P]),
            "orc_conservation": (None, [P, P]),
            "orc_counters": (None, [P, P]),
            "orc_num_threads": (I, []),
            "orc_stream_function": (None, [I, I, P, P]),
            "orc_set_slab": (I, [P, I, I]),
            "orc_collide": (None, [P]),
            "orc_stream": (None, [P, P, P]),
            "orc_post_row": (None, [P, I, P]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Lattice tables (Table I in the column order of T, Eq. Tmatrix).
# --------------------------------------------------------------------------
def d2q9_tables():
    """Return (v [9,2] int, W [9], T [9,9] int, T^{-1} [9,9]) of the oracle."""
    lib = _load()
    v = np.zeros((9, 2), np.int32)
    w = np.zeros(9)
    T = np.zeros((9, 9), np.int32)
    Ti = np.zeros((9, 9))
    lib.orc_d2q9_tables(_ptr(v), _ptr(w), _ptr(T), _ptr(Ti))
    return v, w, T, Ti


def d1q3_tables():
    lib = _load()
    v = np.zeros(3, np.int32)
    w = np.zeros(3)
    lib.orc_d1q3_tables(_ptr(v), _ptr(w))
    return v, w


def tau_from_nu(nu: float) -> float:
    """Eq. (visco-tau) in lattice units: tau = 3 nu + 1/2."""
    return _load().orc_tau_from_nu(nu)


def tau2(tau: float) -> float:
    """Eq. (tau2) as printed: (8 tau - 1) / (2 tau - 1)."""
    return _load().orc_tau2(tau)


# --------------------------------------------------------------------------
# Per-node functions.
# --------------------------------------------------------------------------
def d2q9_feq(rho: float, ux: float, uy: float) -> np.ndarray:
    """Eq. (numerical-plyeqm)."""
    out = np.zeros(9)
    _load().orc_d2q9_feq(float(rho), float(ux), float(uy), _ptr(out))
    return out


def d1q3_feq(rho: float, u: float) -> np.ndarray:
    out = np.zeros(3)
    _load().orc_d1q3_feq(float(rho), float(u), _ptr(out))
    return out


def kld(p, w) -> float:
    """Eq. (discrete_KLD)."""
    p = _f64(p)
    w = _f64(w)
    return _load().orc_kld(len(p), _ptr(p), _ptr(w))


def d2q9_minxent(f, tau: float, nfree: int = 4, tau2_: float | None = None,
                 start: int = START_HYBRID):
    """One MinxEnt collision (Sec. IV.E, single Newton step). -> (fpost, status)."""
    f = _f64(f)
    out = np.zeros(9)
    t2 = tau2(tau) if tau2_ is None else tau2_
    st = _load().orc_d2q9_minxent(_ptr(f), float(tau), float(t2), int(nfree), int(start), _ptr(out))
    return out, st


def d2q9_minxent_converged(f, tau: float, nfree: int = 4, tau2_: float | None = None,
                           gtol: float = 1e-14, maxit: int = 50):
    """Exact constrained KLD minimiser (Eq. minxentLBM-collision). -> (fpost, iters, |grad|)."""
    f = _f64(f)
    out = np.zeros(9)
    g = np.zeros(1)
    t2 = tau2(tau) if tau2_ is None else tau2_
    it = _load().orc_d2q9_minxent_converged(_ptr(f), float(tau), float(t2), int(nfree),
                                             float(gtol), int(maxit), _ptr(out), _ptr(g))
    return out, it, float(g[0])


def d2q9_srt(f, tau: float):
    f = _f64(f)
    out = np.zeros(9)
    st = _load().orc_d2q9_srt(_ptr(f), float(tau), _ptr(out))
    return out, st


def d2q9_mrt(f, tau: float, trt: bool = False, tau2_: float | None = None):
    f = _f64(f)
    out = np.zeros(9)
    t2 = tau2(tau) if tau2_ is None else tau2_
    st = _load().orc_d2q9_mrt(_ptr(f), float(tau), float(t2), int(bool(trt)), _ptr(out))
    return out, st


def d1q3_minxent(f, tau: float):
    f = _f64(f)
    out = np.zeros(3)
    st = _load().orc_d1q3_minxent(_ptr(f), float(tau), _ptr(out))
    return out, st


def d1q3_srt(f, tau: float):
    f = _f64(f)
    out = np.zeros(3)
    st = _load().orc_d1q3_srt(_ptr(f), float(tau), _ptr(out))
    return out, st


def num_threads() -> int:
    return _load().orc_num_threads()


# --------------------------------------------------------------------------
# Lattice simulation (Eq. 2 with the boundary rules of Sec. IV.F).
# --------------------------------------------------------------------------
def stream_function(uy) -> np.ndarray:
    """Sec. IV.I stream function psi = -int_0^x u_y dx per row (lattice
    units; Simpson over pairs of intervals, trapezoid on a last odd one)."""
    uy = _f64(uy)
    ny, nx = uy.shape
    out = np.zeros((ny, nx))
    _load().orc_stream_function(int(nx), int(ny), _ptr(uy), _ptr(out))
    return out


class Sim:
    """One oracle lattice.  Arrays are [y][x] (x fastest); populations [a][y][x]."""

    def __init__(self, lattice: int, nx: int, ny: int, tau: float, bc: int,
                 collision: int = MINXENT4, rho0: float = 1.0, u_lid: float = 0.0):
        self._lib = _load()
        self.lattice, self.nx, self.ny = lattice, nx, ny
        self.q = 9 if lattice == D2Q9 else 3
        self.tau = tau
        h = self._lib.orc_create(int(lattice), int(nx), int(ny), float(tau), int(bc),
                                 int(collision), float(rho0), float(u_lid))
        if not h:
            raise ValueError("oracle rejected the lattice parameters")
        self._h = ctypes.c_void_p(h)

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_start(self, start: int):
        self._lib.orc_set_start(self._h, int(start))

    def set_tau2(self, t2: float):
        self._lib.orc_set_tau2(self._h, float(t2))

    def init(self, rho, ux=None, uy=None):
        n = self.nx * self.ny
        rho = _f64(rho).reshape(n)
        ux = None if ux is None else _f64(ux).reshape(n)
        uy = None if uy is None else _f64(uy).reshape(n)
        self._lib.orc_init(self._h, _ptr(rho), None if ux is None else _ptr(ux),
                           None if uy is None else _ptr(uy))

    def set_f(self, f):
        f = _f64(f).reshape(self.q, self.ny, self.nx)
        self._lib.orc_set_f(self._h, _ptr(f))

    def get_f(self) -> np.ndarray:
        out = np.zeros((self.q, self.ny, self.nx))
        self._lib.orc_get_f(self._h, _ptr(out))
        return out

    def step(self, n: int = 1):
        self._lib.orc_step(self._h, int(n))

    # -- slab form: rows [y_off, y_off + ny) of a lattice of ny_global rows
    def set_slab(self, y_off: int, ny_global: int):
        if self._lib.orc_set_slab(self._h, int(y_off), int(ny_global)) != 0:
            raise ValueError("slab rows outside the lattice")

    def collide(self):
        """First half of Eq. (2): collide every node of this lattice."""
        self._lib.orc_collide(self._h)

    def post_row(self, y: int) -> np.ndarray:
        """Post-collision populations of local row y after collide(), [a][x]."""
        out = np.zeros((self.q, self.nx))
        self._lib.orc_post_row(self._h, int(y), _ptr(out))
        return out

    def stream(self, lo=None, hi=None):
        """Second half of Eq. (2); lo / hi: post-collision rows below the first
        and above the last row ([a][x]), or None for the lattice's own rule."""
        lo = None if lo is None else _f64(lo).reshape(self.q, self.nx)
        hi = None if hi is None else _f64(hi).reshape(self.q, self.nx)
        self._lib.orc_stream(self._h, None if lo is None else _ptr(lo),
                             None if hi is None else _ptr(hi))

    def moments(self):
        rho = np.zeros((self.ny, self.nx))
        ux = np.zeros((self.ny, self.nx))
        uy = np.zeros((self.ny, self.nx))
        self._lib.orc_moments(self._h, _ptr(rho), _ptr(ux), _ptr(uy))
        return rho, ux, uy

    def conservation(self) -> np.ndarray:
        out = np.zeros(3)
        self._lib.orc_conservation(self._h, _ptr(out))
        return out

    def counters(self):
        out = np.zeros(3, np.int64)
        self._lib.orc_counters(self._h, _ptr(out))
        return {"newton_skipped": int(out[0]), "unstable": int(out[1]), "steps": int(out[2])}
