"""lbm_conservation_noalloc: the conservation totals for callers that cannot
allocate device memory (scratch in a fixed array inside the library).

Checked through the C ABI against lbm_conservation_device, the existing entry
point that takes its scratch from the context, on two calls in a row and on
two contexts that share the fixed array.  Collected last (file name), so a
run that stops at the first failure has run every other test already.
"""
import ctypes

import numpy as np
import pytest

from paper_1801_03863_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _dev_totals(fn, lat):
    import torch
    out = torch.full((3 * lat.count,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    code = fn(lat._h, ctypes.c_void_p(out.data_ptr()))
    assert code == lbm.LBM_OK, lbm.lbm_status_string(code)
    lat.stream.synchronize()
    return out.cpu().numpy().reshape(lat.count, 3)


def _check_pair(lat):
    lib = lbm.load()
    ref = _dev_totals(lib.lbm_conservation_device, lat)
    for _ in range(2):  # two calls in a row reuse the same fixed scratch
        got = _dev_totals(lib.lbm_conservation_noalloc, lat)
        scale = np.abs(ref[:, :1]).max()
        assert np.all(np.abs(got - ref) <= TOL * scale), np.abs(got - ref).max()


def test_noalloc_matches_context_scratch():
    members = wl.cavity_ensemble(count=6, seed=4, side_unit=16, side_max_units=5)
    dims = [(m.side, m.side) for m in members]
    rho = np.concatenate([wl.cavity(m.side, noise=1e-6, seed=i)[0].ravel()
                          for i, m in enumerate(members)])
    z = np.zeros_like(rho)
    with lbm.Lattice("d2q9", dims, [m.nu for m in members], "cavity",
                     u_lid=[m.u_lid for m in members], compute="f32", storage="f16") as lat:
        lat.init(rho, z, z)
        lat.step(23)
        _check_pair(lat)
        lat.step(17)
        _check_pair(lat)


def test_noalloc_second_context_sees_no_stale_scratch():
    fields = wl.taylor_green(40, u0=0.05, ny=24)
    with lbm.Lattice("d2q9", [(40, 24)], 0.01, "periodic") as lat:
        lat.init(*fields)
        lat.step(9)
        _check_pair(lat)
    members = wl.tube_ensemble(count=300, seed=1, n_range=(20, 400))
    rho = np.concatenate([wl.tube_fields(m)[0].ravel() for m in members])
    with lbm.Lattice("d1q3", [(m.n, 1) for m in members], [m.nu for m in members],
                     "zero_gradient", compute="f32", storage="f32") as lat:
        lat.init(rho, np.zeros_like(rho))
        lat.step(11)
        _check_pair(lat)


def test_noalloc_rejects_more_instances_than_the_scratch_holds():
    import torch
    n = 4097
    with lbm.Lattice("d1q3", [(8, 1)] * n, [1e-2] * n, "periodic", compute="f32",
                     storage="f32", autotune=False) as lat:
        lat.init(np.ones(8 * n))
        out = torch.empty(3 * n, dtype=torch.float64, device="cuda")
        code = lbm.load().lbm_conservation_noalloc(lat._h, ctypes.c_void_p(out.data_ptr()))
        assert code == lbm.LBM_ERR_ARG
