"""Checkpoint / resume and per-instance ensemble I/O through the C ABI.

Resume: run A takes 2k steps; run B takes k steps, saves its state, loads it
into a new context and takes k more.  A and B must agree bit for bit --
through lbm_save_state / lbm_load_state for every storage type, and through
lbm_get_populations / lbm_set_populations wherever the FP64 populations
round-trip the stored deviations exactly (FP16 and BF16 storage), because the
first step after a load collides with the step kernels' own arithmetic.

Per-instance I/O: lbm_moments_batch / lbm_stream_function_batch of one member
equal that member's slice of the whole-ensemble read-back, and an ensemble
initialised member by member with lbm_init_batch equals one initialised with
lbm_init.
"""
import numpy as np
import pytest

from paper_1801_03863_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu


def _ensemble(count=5, seed=3):
    rng = np.random.default_rng(seed)
    sides = [int(v) for v in rng.integers(3, 40, size=count) * 4]
    sides[0] = 130  # wider than one 128-node tile row, ragged
    nus = list(rng.uniform(0.005, 0.05, size=count))
    ulid = list(rng.uniform(0.05, 0.1, size=count))
    return [(s, s) for s in sides], nus, ulid


def _fields(dims, seed=0):
    rho = np.concatenate([wl.cavity(nx, noise=1e-6, seed=seed + i)[0].ravel()
                          for i, (nx, _) in enumerate(dims)])
    z = np.zeros_like(rho)
    return rho, z, z


def _lattice(dims, nus, ulid, compute, storage, collision="minxent4"):
    return lbm.Lattice("d2q9", dims, nus, "cavity", u_lid=ulid, compute=compute,
                       storage=storage, collision=collision)


@pytest.mark.parametrize("compute,storage", [("f64", "f64"), ("f32", "f32"), ("f32", "f16"),
                                             ("f32", "bf16")])
@pytest.mark.parametrize("collision", ["minxent4", "srt"])
def test_save_load_state_resumes_bit_for_bit(compute, storage, collision):
    dims, nus, ulid = _ensemble()
    fields = _fields(dims)
    k = 37  # odd: the saved state sits in the second buffer
    with _lattice(dims, nus, ulid, compute, storage, collision) as a:
        a.init(*fields)
        a.step(2 * k)
        ref = a.save_state()
        ra = a.moments()
        sa = a.status()
    with _lattice(dims, nus, ulid, compute, storage, collision) as b1:
        b1.init(*fields)
        b1.step(k)
        mid = b1.save_state()
    with _lattice(dims, nus, ulid, compute, storage, collision) as b2:
        b2.load_state(mid)
        b2.step(k)
        got = b2.save_state()
        rb = b2.moments()
        sb = b2.status()
    assert np.array_equal(ref, got)
    for x, y in zip(ra, rb):
        assert np.array_equal(x, y)
    assert sa == sb


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("collision", ["minxent4", "srt", "mrt"])
def test_get_set_populations_resumes_bit_for_bit(storage, collision):
    """FP16/BF16 deviations round-trip exactly through f = W rho0 + d in FP64,
    and the in-place first collision after set_populations uses the step
    kernels' packed FP32x2 arithmetic."""
    dims, nus, ulid = _ensemble(seed=4)
    fields = _fields(dims, seed=10)
    k = 25
    with _lattice(dims, nus, ulid, "f32", storage, collision) as a:
        a.init(*fields)
        a.step(2 * k)
        fa = a.populations()
    with _lattice(dims, nus, ulid, "f32", storage, collision) as b1:
        b1.init(*fields)
        b1.step(k)
        mid = b1.populations()
    with _lattice(dims, nus, ulid, "f32", storage, collision) as b2:
        b2.set_populations(mid)
        assert np.array_equal(b2.populations(), mid)
        b2.step(k)
        fb = b2.populations()
    assert np.array_equal(fa, fb)


@pytest.mark.parametrize("compute,storage,tol", [("f64", "f64", 1e-13), ("f32", "f32", 1e-6)])
def test_get_set_populations_resume_wide_storage(compute, storage, tol):
    """FP32 / FP64 deviations far below W rho0 lose low bits in the FP64
    populations, so this path agrees to that rounding (exact resume: the
    state entry points above)."""
    dims, nus, ulid = _ensemble(seed=5)
    fields = _fields(dims, seed=20)
    k = 25
    with _lattice(dims, nus, ulid, compute, storage) as a:
        a.init(*fields)
        a.step(2 * k)
        fa = a.populations()
    with _lattice(dims, nus, ulid, compute, storage) as b1:
        b1.init(*fields)
        b1.step(k)
        mid = b1.populations()
    with _lattice(dims, nus, ulid, compute, storage) as b2:
        b2.set_populations(mid)
        b2.step(k)
        fb = b2.populations()
    assert np.abs(fa - fb).max() <= tol * np.abs(fa).max()


def test_load_state_rejects_other_layouts():
    dims, nus, ulid = _ensemble()
    fields = _fields(dims)
    with _lattice(dims, nus, ulid, "f32", "f16") as a:
        a.init(*fields)
        a.step(3)
        st = a.save_state()
    other = [(d[0] + 4, d[1]) for d in dims]
    with _lattice(other, nus, ulid, "f32", "f16") as b:
        with pytest.raises(lbm.LBMError) as e:
            b.load_state(st)
        assert e.value.code == lbm.LBM_ERR_ARG
    with _lattice(dims, nus, ulid, "f32", "bf16") as b:
        with pytest.raises(lbm.LBMError):
            b.load_state(st)
    bad = st.copy()
    bad[0] ^= 0xFF  # magic
    with _lattice(dims, nus, ulid, "f32", "f16") as b:
        with pytest.raises(lbm.LBMError):
            b.load_state(bad)


@pytest.mark.parametrize("compute,storage", [("f64", "f64"), ("f32", "f16")])
def test_per_instance_moments_and_stream_function(compute, storage):
    dims, nus, ulid = _ensemble(seed=6)
    fields = _fields(dims, seed=30)
    with _lattice(dims, nus, ulid, compute, storage) as lat:
        lat.init(*fields)
        for check in range(2):  # stored f(t_0), then the pulled f(t_n)
            r, x, y = lat.moments()
            psi = lat.stream_function()
            parts = [lat.split(v) for v in (r, x, y, psi)]
            for i in range(len(dims)):
                ri, xi, yi = lat.moments_instance(i)
                assert np.array_equal(ri, parts[0][i])
                assert np.array_equal(xi, parts[1][i])
                assert np.array_equal(yi, parts[2][i])
                assert np.array_equal(lat.stream_function_instance(i), parts[3][i])
            lat.step(40)


@pytest.mark.parametrize("compute,storage", [("f64", "f64"), ("f32", "bf16")])
def test_init_instance_by_instance_equals_init(compute, storage):
    dims, nus, ulid = _ensemble(seed=7)
    rng = np.random.default_rng(8)
    n = [a * b for a, b in dims]
    rho = [1 + 1e-3 * rng.standard_normal(k) for k in n]
    ux = [0.02 * rng.standard_normal(k) for k in n]
    uy = [0.02 * rng.standard_normal(k) for k in n]
    with _lattice(dims, nus, ulid, compute, storage) as a:
        a.init(np.concatenate(rho), np.concatenate(ux), np.concatenate(uy))
        a.step(20)
        fa = a.populations()
    with _lattice(dims, nus, ulid, compute, storage) as b:
        order = list(range(len(dims)))[::-1]
        for j, i in enumerate(order):
            if j < len(order) - 1:  # not initialised until every instance is
                with pytest.raises(lbm.LBMError):
                    b.step(1)
            b.init_instance(i, rho[i], ux[i], uy[i])
        b.step(20)
        fb = b.populations()
        # mid-run the stored field is post-collision: per-instance init is refused
        with pytest.raises(lbm.LBMError) as e:
            b.init_instance(0, rho[0], ux[0], uy[0])
        assert e.value.code == lbm.LBM_ERR_STATE
    assert np.array_equal(fa, fb)


@pytest.mark.parametrize("compute,storage", [("f64", "f64"), ("f32", "f16")])
def test_page_locked_host_io_equals_staged_io(compute, storage):
    """lbm_init / lbm_moments on page-locked host arrays (kernels read and
    write them in place) give the same values as on ordinary host memory
    (staged through device copies)."""
    import ctypes

    import torch
    dims, nus, ulid = _ensemble(seed=9)
    rho, ux, uy = _fields(dims, seed=40)
    n = rho.size
    pin = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(6)]
    for t, a in zip(pin, (rho, ux, uy)):
        t.numpy()[:] = a
    with _lattice(dims, nus, ulid, compute, storage) as a:
        a.init(rho, ux, uy)
        a.step(30)
        ref = a.moments()
    with _lattice(dims, nus, ulid, compute, storage) as b:
        lib = lbm.load()
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        assert lib.lbm_init(b._h, p(pin[0]), p(pin[1]), p(pin[2])) == lbm.LBM_OK
        b.step(30)
        assert lib.lbm_moments(b._h, p(pin[3]), p(pin[4]), p(pin[5])) == lbm.LBM_OK
        got = [t.numpy().copy() for t in pin[3:]]
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)
