"""The configured workloads at full size, through the C ABI.

At these sizes the oracle cannot run the whole simulation in seconds, so each
test checks (i) one step of every node against the oracle, starting from the
GPU's own state (set into the oracle), and (ii) properties that hold at any
size: conservation, the Taylor-Green decay rate of Eq. (visco-tau), and the
error of the reduced-precision paths against the FP64 path.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1801_03863_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
_VX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
_VY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)


def _one_step_vs_oracle(lat, lattice, nx, ny, nu, bc, u_lid=0.0, tol=1e-12, rho0=1.0):
    """Copy the GPU state f(t_n) into the oracle, take one step on both, and
    compare every population (relative to the largest)."""
    q = 9 if lattice == "d2q9" else 3
    f0 = lat.populations().reshape(q, ny, nx)
    lat.step(1)
    f1 = lat.populations().reshape(q, ny, nx)
    sim = oracle.Sim(oracle.D2Q9 if q == 9 else oracle.D1Q3, nx, ny, oracle.tau_from_nu(nu),
                     {"periodic": oracle.BC_PERIODIC, "cavity": oracle.BC_CAVITY,
                      "zero_gradient": oracle.BC_ZERO_GRADIENT}[bc], rho0=rho0, u_lid=u_lid)
    sim.set_f(f0)
    sim.step(1)
    fo = sim.get_f()
    err = np.abs(f1 - fo).max() / np.abs(fo).max()
    assert err <= tol, err
    return f1


def test_taylor_green_512_fp64():
    """Config: periodic 512^2, u0 = 0.02, nu = 1e-3, FP64; 3000 steps."""
    n, nu = 512, 1e-3
    fields = wl.taylor_green(n, u0=0.02)
    with lbm.Lattice("d2q9", [(n, n)], nu, "periodic") as lat:
        lat.init(*fields)
        c0 = lat.conservation()[0]
        ux0, uy0 = fields[1].ravel(), fields[2].ravel()
        norm = float(ux0 @ ux0 + uy0 @ uy0)
        amps, times = [], []
        # The equilibrium start carries no viscous stress; the first few
        # hundred steps build it up and decay the mode about 16 % faster than
        # the hydrodynamic rate (the FP64 oracle shows the same at 256^2 and
        # 512^2), so the fit starts at step 1000.
        lat.step(1000)
        for k in range(5):
            r, x, y = lat.moments()
            # amplitude of the Taylor-Green velocity mode (projection on the
            # initial pattern): orthogonal to the acoustic modes the
            # equilibrium start excites, it decays as exp(-nu (kx^2 + ky^2) t)
            amps.append(float(x @ ux0 + y @ uy0) / norm)
            times.append(1000 + 500 * k)
            if k < 4:
                lat.step(500)
        c1 = lat.conservation()[0]
        # mass and momentum of a periodic lattice are conserved to rounding
        assert abs(c1[0] - c0[0]) <= 1e-13 * c0[0]
        assert np.abs(c1[1:] - c0[1:]).max() <= 1e-13 * c0[0]
        # velocity decay rate from Eq. (visco-tau): half the energy rate; the
        # oracle's fit over the same window lands within 0.05 % of it
        rate = -np.polyfit(times, np.log(amps), 1)[0]
        assert rate == pytest.approx(0.5 * wl.taylor_green_energy_rate(nu, n), rel=5e-3)
        _one_step_vs_oracle(lat, "d2q9", n, n, nu, "periodic")


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_taylor_green_512_reduced_precision(storage):
    """FP32 compute against the FP64 run after 2000 steps: the velocity field's
    relative error stays at the storage rounding level."""
    n, nu, steps = 512, 1e-3, 2000
    fields = wl.taylor_green(n, u0=0.02)
    res = {}
    for comp, stor in (("f64", "f64"), ("f32", storage)):
        with lbm.Lattice("d2q9", [(n, n)], nu, "periodic", compute=comp, storage=stor) as lat:
            lat.init(*fields)
            lat.step(steps)
            res[comp] = lat.moments()
    r0, x0, y0 = res["f64"]
    r1, x1, y1 = res["f32"]
    u0 = np.sqrt(x0 ** 2 + y0 ** 2).max()
    du = max(np.abs(x1 - x0).max(), np.abs(y1 - y0).max()) / u0
    # per step: FP32 arithmetic (approximate reciprocal and log2, FP32 sums)
    # errs by ~1e-7 W per population, plus the storage rounding u |d| of each
    # deviation (|d| ~ W 3 u0); over 2000 steps, relative to u0: FP32 2e-4,
    # FP16 (u = 2^-11) 3e-2, BF16 (u = 2^-8) 2.5e-1
    bound = {"f32": 2e-4, "f16": 3e-2, "bf16": 2.5e-1}[storage]
    assert du <= bound, du
    assert np.abs(r1 - r0).max() <= 50 * bound * u0 * u0 + 1e-6


def test_cavity_2048_config_errors_at_step_1000():
    """Config: cavity 2048^2, U = 0.1, Re = 5000, FP32 compute with FP16 /
    BF16 / FP32 storage against the FP64 run at step 1000; plus one step of
    the FP64 state against the oracle."""
    side, u = 2048, 0.1
    nu = wl.nu_from_reynolds(5000.0, u, side)
    fields = wl.cavity(side, noise=1e-6, seed=0)
    res = {}
    with lbm.Lattice("d2q9", [(side, side)], nu, "cavity", u_lid=u) as lat:
        lat.init(*fields)
        lat.step(1000)
        res["f64"] = lat.moments()
        assert lat.status()["unstable"] == 0
        _one_step_vs_oracle(lat, "d2q9", side, side, nu, "cavity", u_lid=u)
    for storage in ("f32", "f16", "bf16"):
        with lbm.Lattice("d2q9", [(side, side)], nu, "cavity", u_lid=u, compute="f32",
                         storage=storage) as lat:
            lat.init(*fields)
            lat.step(1000)
            res[storage] = lat.moments()
            assert lat.status()["unstable"] == 0
    r0, x0, y0 = res["f64"]
    errs = {}
    for storage in ("f32", "f16", "bf16"):
        r1, x1, y1 = res[storage]
        errs[storage] = max(np.abs(x1 - x0).max(), np.abs(y1 - y0).max()) / u
    # storage rounding ordering and sizes (relative to the lid speed)
    assert errs["f32"] <= 1e-5, errs
    assert errs["f16"] <= 2e-2, errs
    assert errs["bf16"] <= 1.5e-1, errs
    assert errs["f32"] < errs["f16"] < errs["bf16"], errs


def _fp16_one_step_bound(fo, n_nodes):
    """Per-element bound of one FP32-arithmetic step stored as FP16: the
    FP16 rounding of each deviation (u = 2^-11, times 1.01 for the FP32
    arithmetic before it) plus 2e-6 W_a."""
    dev = np.abs(fo - np.repeat(W9, n_nodes))
    return 2.0 ** -11 * dev * 1.01 + 2e-6 * np.repeat(W9, n_nodes)


@pytest.mark.parametrize("shape", ["smem", "smems", "smemw", "smemd"])
def test_cavity_ensemble_64_one_step_and_conservation(shape, monkeypatch):
    """Config: 64 cavities, FP32 compute, FP16 storage, on the TMA-staged
    kernel with large ("smem") and small ("smems") tiles, 10-warp CTAs
    ("smemw") and the deep ring ("smemd").  One step of every
    node of seven instances against the oracle (from the GPU state): the four
    smallest (side 64: every 64-node unit touches a wall), the two largest
    (1024^2: almost every unit takes the interior fast path) and one whose
    side is not a multiple of 128 (ragged last tile column); and the FP64
    conservation totals against the oracle's sums of the same state."""
    monkeypatch.setenv("LBM_SHAPE", shape)
    members = wl.cavity_ensemble(count=64, seed=0)
    dims = [(m.side, m.side) for m in members]
    rho = np.concatenate([wl.cavity(m.side, noise=1e-6, seed=i)[0].ravel()
                          for i, m in enumerate(members)])
    z = np.zeros_like(rho)
    with lbm.Lattice("d2q9", dims, [m.nu for m in members], "cavity",
                     u_lid=[m.u_lid for m in members], compute="f32", storage="f16") as lat:
        assert lat.launch_shape()["kind"] == {"smem": "smem", "smems": "smem_small",
                                              "smemw": "smem_wide", "smemd": "smem_deep"}[shape]
        lat.init(rho, z, z)
        lat.step(200)
        f0 = lat.populations()
        cons = lat.conservation()
        lat.step(1)
        f1 = lat.populations()
    offs = np.cumsum([0] + [9 * m.side * m.side for m in members])
    by_side = sorted(range(64), key=lambda i: members[i].side)
    ragged = [i for i in by_side if members[i].side % 128 != 0 and members[i].side > 128]
    assert members[by_side[-1]].side == 1024 and ragged
    for i in by_side[:4] + by_side[-2:] + ragged[-1:]:
        m = members[i]
        n = m.side
        a, b = offs[i], offs[i + 1]
        sim = oracle.Sim(oracle.D2Q9, n, n, oracle.tau_from_nu(m.nu), oracle.BC_CAVITY,
                         u_lid=m.u_lid)
        sim.set_f(f0[a:b])
        # the totals against the exactly rounded sums of the same FP64
        # populations (FP16 deviations are exact in them): the reduction adds
        # exact node sums in FP64, so only the FP64 rounding of ~n additions
        # of small partial sums separates the two; the oracle's plain running
        # sum of 9 n populations is less accurate (~9 n u |total|)
        fi = f0[a:b].reshape(9, n * n)
        exact = [math.fsum(fi.ravel()), math.fsum((_VX[:, None] * fi).ravel()),
                 math.fsum((_VY[:, None] * fi).ravel())]
        dev_sum = np.abs(fi - W9[:, None]).sum()
        assert abs(cons[i][0] - exact[0]) <= 1e-14 * exact[0], (cons[i], exact)
        assert np.abs(cons[i][1:] - exact[1:]).max() <= 1e-12 * dev_sum, (cons[i], exact)
        np.testing.assert_allclose(cons[i], sim.conservation(), rtol=1e-10,
                                   atol=1e-10 * dev_sum)
        sim.step(1)
        fo = sim.get_f().ravel()
        tol = _fp16_one_step_bound(fo, n * n)
        assert np.all(np.abs(f1[a:b] - fo) <= tol), (i, n, np.max(np.abs(f1[a:b] - fo) - tol))


@pytest.mark.parametrize("shape", ["smem", "smems", "smemw", "smemd"])
def test_cavity_2048_fp16_one_step_vs_oracle(shape, monkeypatch):
    """Config: cavity 2048^2, U = 0.1, Re = 5000, FP32 compute with FP16
    storage on the TMA-staged kernel.  After 300 steps, one step of every
    node (4.2 M nodes, nearly all through the interior fast path) against the
    oracle's step of the same state (Eq. 2, Sec. IV.E), element by element."""
    monkeypatch.setenv("LBM_SHAPE", shape)
    side, u = 2048, 0.1
    nu = wl.nu_from_reynolds(5000.0, u, side)
    fields = wl.cavity(side, noise=1e-6, seed=0)
    with lbm.Lattice("d2q9", [(side, side)], nu, "cavity", u_lid=u, compute="f32",
                     storage="f16") as lat:
        lat.init(*fields)
        lat.step(300)
        f0 = lat.populations()
        lat.step(1)
        f1 = lat.populations()
        assert lat.status()["unstable"] == 0
    sim = oracle.Sim(oracle.D2Q9, side, side, oracle.tau_from_nu(nu), oracle.BC_CAVITY, u_lid=u)
    sim.set_f(f0)
    sim.step(1)
    fo = sim.get_f().ravel()
    tol = _fp16_one_step_bound(fo, side * side)
    assert np.all(np.abs(f1 - fo) <= tol), np.max(np.abs(f1 - fo) - tol)


def test_tube_ensemble_4096_conservation_fp64_totals():
    """Config: 4096 D1Q3 tubes, FP32 compute.  Per-instance FP64 totals equal
    the oracle's sums of the same state, and one step of sampled tubes matches
    the oracle to FP32 rounding."""
    members = wl.tube_ensemble(count=4096, seed=1)
    dims = [(m.n, 1) for m in members]
    rho = np.concatenate([wl.tube_fields(m)[0].ravel() for m in members])
    with lbm.Lattice("d1q3", dims, [m.nu for m in members], "zero_gradient", compute="f32",
                     storage="f32") as lat:
        lat.init(rho, np.zeros_like(rho))
        c_start = lat.conservation()
        lat.step(2000)
        f0 = lat.populations()
        cons = lat.conservation()
        lat.step(1)
        f1 = lat.populations()
        unstable = [lat.status_instance(i)["unstable"] for i in range(len(members))]
    offs = np.cumsum([0] + [3 * m.n for m in members])
    w3 = np.array([2 / 3, 1 / 6, 1 / 6])
    # the strongest, least viscous tubes blow up (D1Q3 BGK has no entropy
    # limiter): sample both kinds
    stable = [i for i in range(len(members)) if unstable[i] == 0]
    blown = [i for i in range(len(members)) if unstable[i] > 0]
    assert len(stable) >= 6
    checked = 0
    for i in stable[:4] + stable[-2:] + blown[:3]:
        m = members[i]
        a, b = offs[i], offs[i + 1]
        sim = oracle.Sim(oracle.D1Q3, m.n, 1, oracle.tau_from_nu(m.nu), oracle.BC_ZERO_GRADIENT)
        sim.set_f(f0[a:b])
        # NaN totals compare equal: an unstable tube is NaN on both sides
        np.testing.assert_allclose(cons[i], sim.conservation(), rtol=1e-12, atol=1e-9)
        if not np.all(np.isfinite(f0[a:b])):
            # a non-finite state must have been reported for this instance
            assert unstable[i] > 0, i
            continue
        sim.step(1)
        fo = sim.get_f().ravel()
        dev = np.abs(fo - np.repeat(w3, m.n))
        assert np.all(np.abs(f1[a:b] - fo) <= 2.0 ** -24 * dev * 1.01 + 2e-6 * np.repeat(w3, m.n))
        checked += 1
    assert checked >= 6
    # the totals at the start are finite for every tube
    assert np.all(np.isfinite(c_start))
