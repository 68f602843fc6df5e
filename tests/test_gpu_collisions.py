"""Parity of the MinxEnt2, MRT and TRT collision kernels with the FP64 oracle.

MinxEnt2 (Sec. IV.C-E with the extra constraints of Eqs. extraconstraint1/2)
and the MRT / TRT rules of Eq. (mrtcollision) with Table III's rates run in
the same step kernels as MinxEnt4.  FP64: element-by-element agreement within
1e-12 relative; FP32 compute: the storage-rounding bounds of the MinxEnt4
tests; across launch shapes: bitwise.
"""
import numpy as np
import pytest

import oracle
from paper_1801_03863_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
RULES = ["minxent2", "mrt", "trt"]
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _orc_coll(c):
    return {"minxent4": oracle.MINXENT4, "srt": oracle.SRT, "minxent2": oracle.MINXENT2,
            "mrt": oracle.MRT, "trt": oracle.TRT}[c]


def _orc_bc(bc):
    return {"periodic": oracle.BC_PERIODIC, "zero_gradient": oracle.BC_ZERO_GRADIENT,
            "cavity": oracle.BC_CAVITY}[bc]


def _tau2_magic(tau):
    """The magic-parameter reading of Eq. (tau2): (8 tau - 1) / (8 (2 tau - 1))."""
    return (8 * tau - 1) / (8 * (2 * tau - 1))


def _rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _pair(nx, ny, nu, bc, fields, steps, rule, u_lid=0.0, rho0=1.0, tau2_reading="printed"):
    with lbm.Lattice("d2q9", [(nx, ny)], nu, bc, u_lid=u_lid, collision=rule, rho0=rho0,
                     tau2_reading=tau2_reading) as lat:
        lat.init(*fields)
        lat.step(steps)
        gpu = lat.moments() + (lat.populations(), lat.status())
    tau = oracle.tau_from_nu(nu)
    sim = oracle.Sim(oracle.D2Q9, nx, ny, tau, _orc_bc(bc), collision=_orc_coll(rule), rho0=rho0,
                     u_lid=u_lid)
    if tau2_reading == "magic":
        sim.set_tau2(_tau2_magic(tau))
    sim.init(*fields)
    sim.step(steps)
    ro, xo, yo = sim.moments()
    return gpu, (ro.ravel(), xo.ravel(), yo.ravel(), sim.get_f().ravel(), sim.counters())


def _assert_pair(gpu, orc):
    r, x, y, f, st = gpu
    ro, xo, yo, fo, co = orc
    for a, b in ((r, ro), (x, xo), (y, yo)):
        assert _rel(a, b) <= TOL64, _rel(a, b)
        assert np.linalg.norm(a - b) <= TOL64 * np.linalg.norm(b)
    assert _rel(f, fo) <= TOL64
    assert st["unstable"] == co["unstable"] == 0
    assert st["newton_skipped"] == co["newton_skipped"]


# ----------------------------------------------------------------------------
# FP64 parity after many steps.
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny,steps", [(64, 64, 60), (37, 29, 45), (130, 17, 33)])
@pytest.mark.parametrize("rule", RULES)
def test_taylor_green_fp64(rule, nx, ny, steps):
    fields = wl.taylor_green(nx, u0=0.05, ny=ny)
    _assert_pair(*_pair(nx, ny, 0.01, "periodic", fields, steps, rule))


@pytest.mark.parametrize("side,steps,re", [(40, 120, 100.0), (37, 90, 400.0)])
@pytest.mark.parametrize("rule", RULES)
def test_cavity_fp64(rule, side, steps, re):
    u = 0.1
    nu = wl.nu_from_reynolds(re, u, side)
    fields = wl.cavity(side, noise=1e-6, seed=0)
    _assert_pair(*_pair(side, side, nu, "cavity", fields, steps, rule, u_lid=u))


@pytest.mark.parametrize("rule", RULES)
def test_ldss_cavity_density_fp64(rule):
    """Table II LDSS setup: 17 x 17 at rest with rho = 2.7."""
    fields = wl.cavity(17, rho0=2.7)
    _assert_pair(*_pair(17, 17, 0.02, "cavity", fields, 200, rule, u_lid=0.05, rho0=2.7))


@pytest.mark.parametrize("rule", RULES)
def test_paper_shock_tube_fp64(rule):
    """Table II row ST (D2Q9 800 x 4, periodic, tau = 0.5 + 1e-9, 400 steps),
    the setup of Figs. 3-4 that compares these rules.  The state stays
    y-uniform on both sides (every row computes the same values); along x,
    a 1e-15 perturbation grows to at most 1e-13 in 400 steps for these rules,
    so 1e-12 parity is meaningful.  (SRT is left out: at omega ~ 2 it
    amplifies rounding about 1000-fold over the same run.)"""
    nu = 1e-9 / 3.0
    fields = wl.shock_tube_2d(800, 4)
    (r, x, y, f, st), (ro, xo, yo, fo, co) = _pair(800, 4, nu, "periodic", fields, 400, rule)
    assert _rel(r, ro) <= TOL64 and _rel(x, xo) <= TOL64
    assert _rel(f, fo) <= TOL64
    # u_y is zero up to rounding on both sides (the oracle's sums leave ~1e-16)
    assert np.abs(y).max() <= 1e-14 and np.abs(yo).max() <= 1e-14
    assert st["unstable"] == co["unstable"] == 0
    assert st["newton_skipped"] == co["newton_skipped"]


@pytest.mark.parametrize("rule", ["minxent2", "trt"])
def test_tau2_magic_reading_fp64(rule):
    """The alternative reading of Eq. (tau2) changes the heat-flux rate only;
    the oracle takes the same tau2."""
    fields = wl.taylor_green(48, u0=0.05)
    gpu, orc = _pair(48, 48, 0.01, "periodic", fields, 40, rule, tau2_reading="magic")
    _assert_pair(gpu, orc)
    gpu_p, _ = _pair(48, 48, 0.01, "periodic", fields, 40, rule)
    assert _rel(gpu[3], gpu_p[3]) > 1e-9  # the reading matters


# ----------------------------------------------------------------------------
# One step from random states: every node, every population, every boundary.
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("bc", ["periodic", "cavity", "zero_gradient"])
@pytest.mark.parametrize("rule", RULES)
def test_one_step_random_states_fp64(rule, bc):
    nx, ny, nu = 45, 23, 0.02
    f0 = wl.random_populations(9, ny, nx, eps=0.3, seed=12)
    with lbm.Lattice("d2q9", [(nx, ny)], nu, bc, u_lid=0.08, collision=rule) as lat:
        lat.set_populations(f0)
        for k in (1, 2, 3):
            lat.step(1)
            f = lat.populations().reshape(9, ny, nx)
            sim = oracle.Sim(oracle.D2Q9, nx, ny, oracle.tau_from_nu(nu), _orc_bc(bc),
                             collision=_orc_coll(rule), u_lid=0.08)
            sim.set_f(f0)
            sim.step(k)
            assert _rel(f, sim.get_f()) <= TOL64, k


def test_ensemble_mixed_sizes_fp64():
    """One persistent launch over uneven MRT cavities (per-instance rates)."""
    members = wl.cavity_ensemble(count=4, seed=7, side_unit=8, side_max_units=6)
    dims = [(m.side, m.side) for m in members]
    fields = [wl.cavity(m.side, noise=1e-6, seed=i) for i, m in enumerate(members)]
    rho = np.concatenate([f[0].ravel() for f in fields])
    z = np.zeros_like(rho)
    with lbm.Lattice("d2q9", dims, [m.nu for m in members], "cavity",
                     u_lid=[m.u_lid for m in members], collision="mrt") as lat:
        lat.init(rho, z, z)
        lat.step(50)
        f = lat.populations()
    k = 0
    for i, m in enumerate(members):
        n = 9 * m.side * m.side
        sim = oracle.Sim(oracle.D2Q9, m.side, m.side, oracle.tau_from_nu(m.nu), oracle.BC_CAVITY,
                         collision=oracle.MRT, u_lid=m.u_lid)
        sim.init(*fields[i])
        sim.step(50)
        assert _rel(f[k:k + n], sim.get_f()) <= TOL64, i
        k += n


def test_d1q3_rules_are_bgk():
    """On D1Q3 every rule relaxes the single non-conserved moment at 1/tau."""
    n = 301
    fields = wl.shock_tube_1d(n)
    out = {}
    for rule in ("minxent4", "srt", "minxent2", "mrt", "trt"):
        with lbm.Lattice("d1q3", [(n, 1)], 3e-3, "zero_gradient", collision=rule) as lat:
            lat.init(fields[0], fields[1])
            lat.step(120)
            out[rule] = lat.populations()
    for rule in ("srt", "minxent2", "mrt", "trt"):
        assert np.array_equal(out[rule], out["minxent4"]), rule
    sim = oracle.Sim(oracle.D1Q3, n, 1, oracle.tau_from_nu(3e-3), oracle.BC_ZERO_GRADIENT,
                     collision=oracle.SRT)
    sim.init(fields[0], fields[1])
    sim.step(120)
    assert _rel(out["srt"], sim.get_f()) <= TOL64


# ----------------------------------------------------------------------------
# FP32 compute: launch shapes bitwise, storage rounding against the oracle.
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("bc,dims", [("periodic", [(37, 29)]), ("cavity", [(133, 133), (64, 64)]),
                                     ("zero_gradient", [(264, 5)])])
@pytest.mark.parametrize("rule", RULES)
def test_launch_shapes_agree_bitwise(rule, storage, bc, dims, monkeypatch):
    nus = [0.01 + 0.002 * i for i in range(len(dims))]
    parts = [wl.random_populations(9, ny, nx, eps=0.2, seed=3 + i).ravel()
             for i, (nx, ny) in enumerate(dims)]
    f0 = np.concatenate(parts)
    chunk = "2,16,8" if storage == "f32" else "4,8,16"
    out = {}
    for s in (chunk, "smem", "smems", "smemw", "smemd"):
        monkeypatch.setenv("LBM_SHAPE", s)
        with lbm.Lattice("d2q9", dims, nus, bc, u_lid=0.07, compute="f32", storage=storage,
                         collision=rule) as lat:
            lat.set_populations(f0)
            lat.step(21)
            out[s] = (lat.populations(), lat.status())
    for s in ("smem", "smems", "smemw", "smemd"):
        assert out[s][1] == out[chunk][1], s
        assert np.array_equal(out[s][0], out[chunk][0]), s


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("rule", RULES)
def test_reduced_precision_one_step_every_node(rule, storage):
    """From a state exactly representable in every storage type, one step
    differs from the oracle by FP32 arithmetic (bounded by 2e-6 W) plus the
    rounding of each deviation to storage (u |d|)."""
    import torch
    nx, ny, nu = 64, 24, 0.02
    f0 = wl.random_populations(9, ny, nx, eps=0.2, seed=5)
    w = W9[:, None, None]
    dev0 = torch.tensor(f0 - w).to(torch.bfloat16).to(torch.float64).numpy()
    f0 = w + dev0
    with lbm.Lattice("d2q9", [(nx, ny)], nu, "periodic", compute="f32", storage=storage,
                     collision=rule) as lat:
        lat.set_populations(f0)
        lat.step(1)
        f = lat.populations().reshape(9, ny, nx)
    sim = oracle.Sim(oracle.D2Q9, nx, ny, oracle.tau_from_nu(nu), oracle.BC_PERIODIC,
                     collision=_orc_coll(rule))
    sim.set_f(f0)
    sim.step(1)
    fo = sim.get_f()
    u = {"f32": 2.0 ** -24, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}[storage]
    tol = u * np.abs(fo - w) * 1.01 + 2e-6 * w
    assert np.all(np.abs(f - fo) <= tol), np.max(np.abs(f - fo) - tol)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
@pytest.mark.parametrize("rule", ["minxent4", "minxent2"])
def test_negative_start_pair_skips_newton(rule, storage):
    """Reading C-NEG when two opposite start probabilities are negative
    together: a uniform state at rest with a strongly negative xx-stress and
    tau = 300.5 has y_1 = y_3 ~ -0.2 (all other y positive) for several steps.
    Their product is positive, so a gradient formed from logarithms of
    products (the FP32 MinxEnt2 path) only sees the sign through its
    explicit sign-bit test.  Every node must skip its Newton step and keep
    p^start (which has negative populations, so it also counts as unstable),
    exactly as the oracle does."""
    W9_ = W9
    dev = np.array([0, -1, 2, -1, 2, 0, 0, 0, 0.0])
    nx, ny, nu, steps = 24, 10, 100.0, 5
    f0 = np.repeat(W9_ * (1 + dev), nx * ny).reshape(9, ny, nx)
    compute = "f64" if storage == "f64" else "f32"
    with lbm.Lattice("d2q9", [(nx, ny)], nu, "periodic", compute=compute, storage=storage,
                     collision=rule) as lat:
        lat.set_populations(f0)
        lat.step(steps)
        f = lat.populations().reshape(9, ny, nx)
        st = lat.status()
    sim = oracle.Sim(oracle.D2Q9, nx, ny, oracle.tau_from_nu(nu), oracle.BC_PERIODIC,
                     collision=_orc_coll(rule))
    sim.set_f(f0)
    sim.step(steps)
    co = sim.counters()
    assert co["newton_skipped"] == nx * ny * steps
    assert st["newton_skipped"] == co["newton_skipped"], (st, co)
    assert st["unstable"] == co["unstable"], (st, co)
    fo = sim.get_f()
    if storage == "f64":
        assert _rel(f, fo) <= TOL64
    else:
        u = {"f32": 2.0 ** -24, "f16": 2.0 ** -11}[storage]
        w = W9_[:, None, None]
        # a few FP32 steps on O(1) values plus the storage rounding of each deviation
        tol = steps * (u * np.abs(fo - w) * 1.01 + 4e-7 * w)
        assert np.all(np.abs(f - fo) <= tol), np.max(np.abs(f - fo) - tol)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("rule", ["minxent4", "minxent2"])
def test_negative_post_collision_population_is_counted(rule, storage):
    """The criterion of Sec. IV.H on nodes that took their Newton step: in a
    strongly perturbed random state (eps 0.9, seed 2, nu 0.2) some nodes
    have a positive start point but a negative post-collision population
    (MinxEnt4: 4 such nodes; MinxEnt2: 1, besides 24 skipped nodes), and no
    post-collision population lies within 3e-5 of zero.  The kernel decides
    the sign on its FP32 result, before the rounding to storage, so it must
    count the same nodes as the oracle."""
    import torch
    nx, ny, nu = 48, 24, 0.2
    w = W9[:, None, None]
    f0 = wl.random_populations(9, ny, nx, eps=0.9, seed=2)
    f0 = w + torch.tensor(f0 - w).to(torch.bfloat16).to(torch.float64).numpy()
    with lbm.Lattice("d2q9", [(nx, ny)], nu, "periodic", compute="f32", storage=storage,
                     collision=rule) as lat:
        lat.set_populations(f0)
        lat.step(1)
        st = lat.status()
    sim = oracle.Sim(oracle.D2Q9, nx, ny, oracle.tau_from_nu(nu), oracle.BC_PERIODIC,
                     collision=_orc_coll(rule))
    sim.set_f(f0)
    sim.step(1)
    co = sim.counters()
    assert co["unstable"] > co["newton_skipped"]  # the premise: common-path negatives exist
    assert st["newton_skipped"] == co["newton_skipped"], (st, co)
    assert st["unstable"] == co["unstable"], (st, co)
