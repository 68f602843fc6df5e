"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 path: element-by-element agreement of rho and u (and of the
populations) within 1e-12 relative after N steps -- the FP64 kernel and the
oracle evaluate the same algorithm in different but algebraically equal
forms, so they differ by rounding only.
Reduced precision (FP32 compute, FP32/FP16/BF16 storage): errors against the
oracle within bounds derived from the storage rounding unit (see
``_storage_tol``).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1801_03863_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() / scale, np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _orc_bc(bc):
    return {"periodic": oracle.BC_PERIODIC, "zero_gradient": oracle.BC_ZERO_GRADIENT,
            "cavity": oracle.BC_CAVITY}[bc]


def _orc_coll(c):
    return {"minxent4": oracle.MINXENT4, "srt": oracle.SRT}[c]


def _run_pair(lattice, nx, ny, nu, bc, fields, steps, collision="minxent4", u_lid=0.0, rho0=1.0,
              compute="f64", storage=None, autotune=True):
    q = 9 if lattice == "d2q9" else 3
    with lbm.Lattice(lattice, [(nx, ny)], nu, bc, u_lid=u_lid, compute=compute, storage=storage,
                     collision=collision, rho0=rho0, autotune=autotune) as lat:
        lat.init(*fields)
        lat.step(steps)
        r, x, y = lat.moments()
        f = lat.populations().reshape(q, ny, nx)
        st = lat.status()
    sim = oracle.Sim(oracle.D2Q9 if q == 9 else oracle.D1Q3, nx, ny, oracle.tau_from_nu(nu),
                     _orc_bc(bc), collision=_orc_coll(collision), rho0=rho0, u_lid=u_lid)
    sim.init(*fields)
    sim.step(steps)
    ro, xo, yo = sim.moments()
    return (r.reshape(ny, nx), x.reshape(ny, nx), None if y is None else y.reshape(ny, nx), f, st), \
        (ro, xo, yo, sim.get_f(), sim.counters())


def _assert_fp64(gpu, orc, mask=None):
    r, x, y, f, st = gpu
    ro, xo, yo, fo, co = orc
    sel = (slice(None),) if mask is None else (mask,)
    for a, b in ((r, ro), (x, xo)) + (((y, yo),) if y is not None else ()):
        linf, l2 = _rel(a[sel], b[sel])
        assert linf <= TOL64 and l2 <= TOL64, (linf, l2)
    linf, _ = _rel(f[(slice(None),) + sel] if mask is not None else f,
                   fo[(slice(None),) + sel] if mask is not None else fo)
    assert linf <= TOL64, linf
    assert st["unstable"] == co["unstable"] == 0
    assert st["newton_skipped"] == co["newton_skipped"]


# ----------------------------------------------------------------------------
# FP64 parity on the configured workloads and ragged / multi-tile shapes.
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny,steps", [(64, 64, 60), (37, 29, 45), (8, 3, 20), (130, 17, 33)])
@pytest.mark.parametrize("collision", ["minxent4", "srt"])
def test_taylor_green_fp64(nx, ny, steps, collision):
    fields = wl.taylor_green(nx, u0=0.05, ny=ny)
    gpu, orc = _run_pair("d2q9", nx, ny, 0.01, "periodic", fields, steps, collision=collision)
    _assert_fp64(gpu, orc)


@pytest.mark.parametrize("side,steps,re", [(40, 120, 100.0), (37, 90, 400.0), (64, 50, 1000.0)])
def test_cavity_fp64(side, steps, re):
    u = 0.1
    nu = wl.nu_from_reynolds(re, u, side)
    fields = wl.cavity(side, rho0=1.0, noise=1e-6, seed=0)
    gpu, orc = _run_pair("d2q9", side, side, nu, "cavity", fields, steps, u_lid=u)
    _assert_fp64(gpu, orc)


def test_cavity_paper_density_fp64():
    """Table II LDSS setup: rho = 2.7 at rest, 17 x 17."""
    side, u = 17, 0.05
    fields = wl.cavity(side, rho0=2.7)
    gpu, orc = _run_pair("d2q9", side, side, 0.02, "cavity", fields, 200, u_lid=u, rho0=2.7)
    _assert_fp64(gpu, orc)


def test_shock_tube_d1q3_full_config():
    """800 nodes, rho 1 | 0.5, nu = 1e-3, zero-gradient ends, 400 steps."""
    fields = wl.shock_tube_1d(800)
    gpu, orc = _run_pair("d1q3", 800, 1, 1e-3, "zero_gradient", (fields[0], fields[1]), 400)
    _assert_fp64(gpu, orc)


@pytest.mark.parametrize("n", [203, 1001])
def test_shock_tube_d1q3_ragged(n):
    fields = wl.shock_tube_1d(n)
    gpu, orc = _run_pair("d1q3", n, 1, 3e-3, "zero_gradient", (fields[0], fields[1]), 150)
    _assert_fp64(gpu, orc)


def test_shock_tube_d2q9_paper_form():
    """Table II row ST: D2Q9 (800, 4), periodic, tau = 0.5 + 1e-9, 400 steps."""
    nu = 1e-9 / 3.0
    fields = wl.shock_tube_2d(800, 4)
    gpu, orc = _run_pair("d2q9", 800, 4, nu, "periodic", fields, 400)
    r, x, y, f, st = gpu
    ro, xo, yo, fo, co = orc
    assert st["newton_skipped"] == co["newton_skipped"]
    assert st["unstable"] == co["unstable"]
    linf, l2 = _rel(r, ro)
    assert linf <= TOL64 and l2 <= TOL64, (linf, l2)
    linf, _ = _rel(x, xo)
    assert linf <= TOL64


# ----------------------------------------------------------------------------
# One step from random populations: every node, every population.
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("bc", ["periodic", "cavity", "zero_gradient"])
def test_one_step_random_states_fp64(bc):
    nx, ny = 45, 23
    f0 = wl.random_populations(9, ny, nx, eps=0.3, seed=12)
    with lbm.Lattice("d2q9", [(nx, ny)], 0.02, bc, u_lid=0.08) as lat:
        lat.set_populations(f0)
        for k in (1, 2, 3):
            lat.step(1)
            f = lat.populations().reshape(9, ny, nx)
            sim = oracle.Sim(oracle.D2Q9, nx, ny, oracle.tau_from_nu(0.02), _orc_bc(bc),
                             u_lid=0.08)
            sim.set_f(f0)
            sim.step(k)
            linf, _ = _rel(f, sim.get_f())
            assert linf <= TOL64, (k, linf)


# Lattices of one to a few nodes per side, as one uneven ensemble: every node
# is an edge node, tile rows are mostly padding, and x shifts wrap or clamp
# onto the node itself.  Cavities need an interior node (3 x 3 at least).
_TINY = {"periodic": [(1, 1), (2, 3), (5, 2), (1, 9), (9, 1), (3, 3)],
         "zero_gradient": [(1, 1), (2, 3), (5, 2), (1, 9), (9, 1), (3, 3)],
         "cavity": [(3, 3), (4, 3), (3, 5), (17, 4)]}


def _tiny_state(dims):
    parts = [wl.random_populations(9, ny, nx, eps=0.2, seed=5 + i)
             for i, (nx, ny) in enumerate(dims)]
    return parts, np.concatenate([p.ravel() for p in parts])


@pytest.mark.parametrize("bc", ["periodic", "zero_gradient", "cavity"])
def test_tiny_lattices_fp64_match_oracle(bc):
    dims = _TINY[bc]
    parts, f0 = _tiny_state(dims)
    steps = 9
    with lbm.Lattice("d2q9", dims, 0.02, bc, u_lid=0.08) as lat:
        lat.set_populations(f0)
        lat.step(steps)
        f = lat.populations()
    k = 0
    for i, (nx, ny) in enumerate(dims):
        n = 9 * nx * ny
        sim = oracle.Sim(oracle.D2Q9, nx, ny, oracle.tau_from_nu(0.02), _orc_bc(bc), u_lid=0.08)
        sim.set_f(parts[i])
        sim.step(steps)
        linf, _ = _rel(f[k:k + n], sim.get_f())
        assert linf <= TOL64, (bc, nx, ny, linf)
        k += n


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("bc", ["periodic", "zero_gradient", "cavity"])
def test_tiny_lattices_kernels_agree_bitwise(storage, bc, monkeypatch):
    """The TMA kernel (both tile geometries) and the register-chunk kernel
    agree bit for bit on the tiny ensemble."""
    dims = _TINY[bc]
    _, f0 = _tiny_state(dims)
    chunk = "2,16,8" if storage == "f32" else "4,8,16"
    out = {}
    for s in (chunk, "smem", "smems"):
        monkeypatch.setenv("LBM_SHAPE", s)
        with lbm.Lattice("d2q9", dims, 0.02, bc, u_lid=0.08, compute="f32",
                         storage=storage) as lat:
            lat.set_populations(f0)
            lat.step(9)
            out[s] = (lat.populations(), lat.status())
    for s in ("smem", "smems"):
        assert out[s][1] == out[chunk][1], s
        assert np.array_equal(out[s][0], out[chunk][0]), s


# ----------------------------------------------------------------------------
# Ensembles: one persistent launch over uneven instances.
# ----------------------------------------------------------------------------
def test_cavity_ensemble_fp64():
    members = wl.cavity_ensemble(count=5, seed=3, side_unit=8, side_max_units=6)
    dims = [(m.side, m.side) for m in members]
    nus = [m.nu for m in members]
    uls = [m.u_lid for m in members]
    fields = [wl.cavity(m.side, noise=1e-6, seed=i) for i, m in enumerate(members)]
    rho = np.concatenate([f[0].ravel() for f in fields])
    z = np.zeros_like(rho)
    steps = 70
    with lbm.Lattice("d2q9", dims, nus, "cavity", u_lid=uls) as lat:
        lat.init(rho, z, z)
        lat.step(steps)
        r, x, y = lat.moments()
        cons = lat.conservation()
    k = 0
    for i, m in enumerate(members):
        n = m.side * m.side
        sim = oracle.Sim(oracle.D2Q9, m.side, m.side, oracle.tau_from_nu(m.nu), oracle.BC_CAVITY,
                         u_lid=m.u_lid)
        sim.init(*fields[i])
        sim.step(steps)
        ro, xo, yo = sim.moments()
        for a, b in ((r[k:k + n], ro), (x[k:k + n], xo), (y[k:k + n], yo)):
            assert _rel(a, b)[0] <= TOL64
        np.testing.assert_allclose(cons[i], sim.conservation(), rtol=1e-12, atol=1e-12 * n)
        k += n


def test_tube_ensemble_fp64_conservation():
    """Uneven D1Q3 tubes in one launch.  At nu ~ 1e-5 with a 4:1 density jump
    BGK (= MinxEnt on D1Q3) overshoots at the shock and some populations go
    negative; the status counters must match the oracle's instance by
    instance, and the (finite) fields must still agree."""
    members = wl.tube_ensemble(count=12, seed=1, n_range=(50, 900))
    dims = [(m.n, 1) for m in members]
    fields = [wl.tube_fields(m) for m in members]
    rho = np.concatenate([f[0].ravel() for f in fields])
    steps = 64
    with lbm.Lattice("d1q3", dims, [m.nu for m in members], "zero_gradient") as lat:
        lat.init(rho, np.zeros_like(rho))
        lat.step(steps)
        r, x, _ = lat.moments(allow_unstable=True)
        cons = lat.conservation()
        per = [lat.status_instance(i) for i in range(len(members))]
    k = 0
    for i, m in enumerate(members):
        sim = oracle.Sim(oracle.D1Q3, m.n, 1, oracle.tau_from_nu(m.nu), oracle.BC_ZERO_GRADIENT)
        sim.init(*fields[i])
        sim.step(steps)
        ro, xo, _ = sim.moments()
        assert per[i]["unstable"] == sim.counters()["unstable"], i
        # An instance that went unstable (negative populations, Sec. IV.H)
        # amplifies rounding differences step by step; the 1e-12 bound applies
        # to the stable ones, the unstable ones must still agree to 1e-8.
        tol = TOL64 if per[i]["unstable"] == 0 else 1e-8
        assert _rel(r[k:k + m.n], ro)[0] <= tol, (i, per[i])
        assert np.abs(x[k:k + m.n] - xo.ravel()).max() <= tol * max(np.abs(xo).max(), 1e-3)
        co = sim.conservation()
        assert abs(cons[i, 0] - co[0]) <= 1e-12 * co[0]
        assert abs(cons[i, 1] - co[1]) <= 1e-12 * co[0]
        k += m.n


# ----------------------------------------------------------------------------
# Conservation reduction, launch-shape independence, status reporting.
# ----------------------------------------------------------------------------
_VX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
_VY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("bc", ["cavity", "periodic"])
def test_conservation_reduced_storage_matches_state_sums(storage, bc):
    """The FP64 totals of the reduction equal the sums of the same state read
    back as FP64 populations, right after a load (stored f(t_n)) and after
    steps (the pulled f(t_n)), for an instance taller than the 64 partial
    rows of the reduction and one shorter.  Every storage type agrees to
    FP64 rounding: FP32 and BF16 values sum in compensated FP32 pairs, FP16
    node sums are exact integers of 2^-24 units (no FP32 rounding anywhere)."""
    dims = [(150, 133), (37, 20)]
    f0 = np.concatenate([wl.random_populations(9, ny, nx, eps=0.2, seed=11 + i).ravel()
                         for i, (nx, ny) in enumerate(dims)])
    with lbm.Lattice("d2q9", dims, [0.01, 0.02], bc, u_lid=0.05, compute="f32",
                     storage=storage) as lat:
        lat.set_populations(f0)
        checks = [(lat.conservation(), lat.populations())]
        lat.step(7)
        checks.append((lat.conservation(), lat.populations()))
    for cons, f in checks:
        k = 0
        for i, (nx, ny) in enumerate(dims):
            fi = f[k:k + 9 * nx * ny].reshape(9, ny * nx)
            k += 9 * nx * ny
            want = np.array([fi.sum(), (_VX[:, None] * fi).sum(), (_VY[:, None] * fi).sum()])
            assert np.abs(cons[i] - want).max() <= 2e-12 * want[0], (storage, bc, i)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_conservation_propagates_non_finite_values(storage):
    """A NaN or an infinity in an instance's state makes that instance's
    totals NaN / infinite (the reduction's fast paths hand such nodes to the
    FP64 path); the other instances' totals stay finite and exact."""
    dims = [(40, 30), (33, 21), (25, 25)]
    f0 = np.concatenate([wl.random_populations(9, ny, nx, eps=0.05, seed=31 + i).ravel()
                         for i, (nx, ny) in enumerate(dims)])
    base = [0, 9 * 40 * 30, 9 * (40 * 30 + 33 * 21)]
    f0[base[0] + 5 * 40 * 30 + 7] = np.nan      # instance 0: a NaN
    f0[base[1] + 2 * 33 * 21 + 100] = np.inf    # instance 1: +inf, pulled along +y
    with lbm.Lattice("d2q9", dims, 0.02, "periodic", compute="f32", storage=storage) as lat:
        lat.set_populations(f0)
        cons = lat.conservation()
        f = lat.populations()
    assert np.isnan(cons[0, 0])
    assert np.isinf(cons[1, 0]) and cons[1, 0] > 0 and np.isinf(cons[1, 2])
    fi = f[base[2]:].reshape(9, 25 * 25)
    want = np.array([fi.sum(), (_VX[:, None] * fi).sum(), (_VY[:, None] * fi).sum()])
    assert np.all(np.isfinite(cons[2])) and np.abs(cons[2] - want).max() <= 2e-12 * want[0]


def test_conservation_periodic_is_exact_and_reproducible():
    n = 96
    fields = wl.taylor_green(n, u0=0.05)
    with lbm.Lattice("d2q9", [(n, n)], 0.005, "periodic") as lat:
        lat.init(*fields)
        c0 = lat.conservation()
        lat.step(100)
        c1 = lat.conservation()
        c1b = lat.conservation()
    assert np.array_equal(c1, c1b)  # fixed summation order
    assert abs(c1[0, 0] - c0[0, 0]) <= 1e-13 * c0[0, 0]
    assert np.abs(c1[0, 1:] - c0[0, 1:]).max() <= 1e-13 * c0[0, 0]
    sim = oracle.Sim(oracle.D2Q9, n, n, oracle.tau_from_nu(0.005), oracle.BC_PERIODIC)
    sim.init(*fields)
    sim.step(100)
    np.testing.assert_allclose(c1[0], sim.conservation(), rtol=1e-12, atol=1e-12 * n * n)


@pytest.mark.parametrize("storage", ["f64", "f16"])
def test_launch_shapes_agree_bitwise(storage, monkeypatch):
    nx, ny = 72, 40
    fields = wl.taylor_green(nx, u0=0.05, ny=ny)
    compute = "f64" if storage == "f64" else "f32"
    shapes = ["2,4,32", "2,16,8", "2,64,4"] if storage == "f64" else \
        ["4,8,16", "8,4,32", "8,32,8", "smem", "smems", "smemw", "smemd"]
    ref = None
    for s in shapes:
        monkeypatch.setenv("LBM_SHAPE", s)
        with lbm.Lattice("d2q9", [(nx, ny)], 0.01, "periodic", compute=compute,
                         storage=storage) as lat:
            sh = lat.launch_shape()
            if s.startswith("smem"):
                assert sh["kind"] == {"smem": "smem", "smems": "smem_small", "smemw": "smem_wide",
                                     "smemd": "smem_deep"}[s]
                assert sh["V"] == 2
            else:
                assert sh["V"] == int(s.split(",")[0]) and sh["kind"] == "chunks"
            lat.init(*fields)
            lat.step(37)
            f = lat.populations()
        if ref is None:
            ref = f
        else:
            assert np.array_equal(f, ref), s


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("bc,dims", [("periodic", [(37, 29)]), ("periodic", [(300, 9)]),
                                     ("cavity", [(70, 50)]), ("cavity", [(133, 133), (64, 64)]),
                                     ("zero_gradient", [(45, 23)]), ("zero_gradient", [(264, 5)])])
def test_smem_kernel_matches_chunk_kernel(storage, bc, dims, monkeypatch):
    """The shared-memory staged kernel and the register-chunk kernel run the
    same FP32 arithmetic in the same order, so they agree bit for bit, over
    ragged widths, multi-tile rows, every boundary kind and ensembles."""
    nus = [0.01 + 0.002 * i for i in range(len(dims))]
    f0 = np.concatenate([wl.random_populations(9, ny, nx, eps=0.2, seed=3 + i).reshape(9, -1)
                         for i, (nx, ny) in enumerate(dims)], axis=1)
    # per-instance [a][y][x] blocks, concatenated
    parts, k = [], 0
    for nx, ny in dims:
        parts.append(f0[:, k:k + nx * ny].ravel())
        k += nx * ny
    f0 = np.concatenate(parts)
    out = {}
    for s in ("4,8,16", "smem", "smems", "smemw", "smemd"):
        monkeypatch.setenv("LBM_SHAPE", s if storage != "f32" or s.startswith("smem") else "2,16,8")
        with lbm.Lattice("d2q9", dims, nus, bc, u_lid=0.07, compute="f32", storage=storage) as lat:
            lat.set_populations(f0)
            lat.step(21)
            out[s] = (lat.populations(), lat.status())
    for s in ("smem", "smems", "smemw", "smemd"):
        assert out[s][1] == out["4,8,16"][1], s
        assert np.array_equal(out[s][0], out["4,8,16"][0]), s


def test_unstable_node_is_reported():
    nx, ny = 24, 16
    f0 = wl.random_populations(9, ny, nx, eps=0.2, seed=2)
    f0[3, 5, 7] = np.nan
    with lbm.Lattice("d2q9", [(nx, ny)], 0.01, "periodic") as lat:
        lat.set_populations(f0)
        lat.step(2)
        st = lat.status()
        assert st["unstable"] >= 1
        with pytest.raises(lbm.LBMError) as e:
            lat.moments()
        assert e.value.code == lbm.LBM_ERR_UNSTABLE
        r, _, _ = lat.moments(allow_unstable=True)
        assert np.isnan(r).any()


def test_step_before_init_is_a_state_error():
    with lbm.Lattice("d2q9", [(16, 16)], 0.01, "periodic") as lat:
        with pytest.raises(lbm.LBMError) as e:
            lat.step(1)
        assert e.value.code == lbm.LBM_ERR_STATE


def test_library_owned_memory_path():
    n = 32
    fields = wl.taylor_green(n, u0=0.05)
    with lbm.Lattice("d2q9", [(n, n)], 0.01, "periodic", torch_memory=False) as lat:
        lat.init(*fields)
        lat.step(20)
        r, _, _ = lat.moments()
    sim = oracle.Sim(oracle.D2Q9, n, n, oracle.tau_from_nu(0.01), oracle.BC_PERIODIC)
    sim.init(*fields)
    sim.step(20)
    assert _rel(r, sim.moments()[0])[0] <= TOL64


def test_device_io_matches_host_io():
    import torch
    n = 48
    fields = wl.taylor_green(n, u0=0.05)
    with lbm.Lattice("d2q9", [(n, n)], 0.01, "periodic") as lat:
        dev = [torch.tensor(a.ravel(), dtype=torch.float64, device="cuda") for a in fields]
        torch.cuda.synchronize()
        lat.init_device(*dev)
        lat.step(10)
        out = [torch.empty(n * n, dtype=torch.float64, device="cuda") for _ in range(3)]
        lat.moments_device(*out)
        lat.stream.synchronize()
        r_dev = out[0].cpu().numpy()
        r_host, _, _ = lat.moments()
    assert np.array_equal(r_dev, r_host)


# ----------------------------------------------------------------------------
# Reduced precision against the FP64 oracle.
# ----------------------------------------------------------------------------
def _storage_tol(storage):
    """Unit roundoff u of the storage type (round to nearest even):
    |round(x) - x| <= u |x| with u = 2^-24 (FP32), 2^-11 (FP16), 2^-8 (BF16)."""
    return {"f32": 2.0 ** -24, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}[storage]


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_reduced_precision_taylor_green(storage):
    n, steps, nu, u0 = 64, 200, 0.01, 0.05
    fields = wl.taylor_green(n, u0=u0)
    gpu, orc = _run_pair("d2q9", n, n, nu, "periodic", fields, steps, compute="f32",
                         storage=storage)
    r, x, y, f, st = gpu
    ro, xo, yo, fo, co = orc
    assert st["unstable"] == 0
    # deviations are O(W u0); their rounding unit bounds the per-step error
    eps = _storage_tol(storage)
    bound_u = 50 * eps * u0 + 2e-6 * u0
    bound_r = 50 * eps * 3 * u0 * u0 + 2e-6
    assert np.abs(x - xo).max() <= bound_u, np.abs(x - xo).max()
    assert np.abs(y - yo).max() <= bound_u
    assert np.abs(r - ro).max() <= bound_r, np.abs(r - ro).max()


@pytest.mark.parametrize("shape", ["auto", "smem", "smems", "smemw", "smemd"])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_reduced_precision_one_step_every_node(storage, shape, monkeypatch):
    """One step from an FP16-representable state: the only differences are
    FP32 arithmetic and the final rounding of each deviation to storage."""
    nx, ny = 64, 24
    f0 = wl.random_populations(9, ny, nx, eps=0.2, seed=5)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    # make the start exactly representable in every storage type
    import torch
    dev0 = f0 - w
    dev0 = torch.tensor(dev0).to(torch.bfloat16).to(torch.float64).numpy()
    f0 = w + dev0
    if shape != "auto":
        monkeypatch.setenv("LBM_SHAPE", shape)
    with lbm.Lattice("d2q9", [(nx, ny)], 0.02, "periodic", compute="f32", storage=storage) as lat:
        lat.set_populations(f0)
        lat.step(1)
        f = lat.populations().reshape(9, ny, nx)
    sim = oracle.Sim(oracle.D2Q9, nx, ny, oracle.tau_from_nu(0.02), oracle.BC_PERIODIC)
    sim.set_f(f0)
    sim.step(1)
    fo = sim.get_f()
    dev_o = fo - w
    # storage rounding of each deviation (u |d|, 1% slack for |d_gpu| vs |d|)
    # plus FP32 arithmetic on terms of size W (a few ulps of W, bounded by 2e-6 W)
    tol = _storage_tol(storage) * np.abs(dev_o) * 1.01 + 2e-6 * w
    assert np.all(np.abs(f - fo) <= tol), np.max(np.abs(f - fo) - tol)
