"""The C ABI library: it loads, exports every entry point include/lbm.h
declares, and validates arguments before touching a device (CPU tests)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1801_03863_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return lbm.load()


def test_every_declared_symbol_is_exported(lib):
    names = _header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(lbm.EXPORTS)


def test_status_strings(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        s = lbm.lbm_status_string(code)
        assert s and "unknown" not in s
    assert "unknown" in lbm.lbm_status_string(-99)


def test_default_opts(lib):
    o = lbm.lbm_default_opts()
    assert (o.compute, o.storage, o.collision, o.autotune, o.rho0) == (0, 0, 0, 1, 1.0)


def test_required_bytes_scales_with_storage(lib):
    o = lbm.lbm_default_opts()
    b64 = lbm.lbm_required_bytes(lbm.LBM_D2Q9, [512, 512], o)
    o.compute, o.storage = lbm.LBM_F32, lbm.LBM_F16
    b16 = lbm.lbm_required_bytes(lbm.LBM_D2Q9, [512, 512], o)
    # two population buffers of 9 planes; FP64 staging dominates the rest
    assert b64 >= 2 * 9 * 512 * 512 * 8
    assert b16 >= 2 * 9 * 512 * 512 * 2
    assert b64 - b16 >= 2 * 9 * 512 * 512 * 6


@pytest.mark.parametrize("lat,dims,comp,stor", [
    (3, [8, 8], 0, 0),                 # bad lattice
    (1, [8, 2], 0, 0),                 # D1Q3 needs ny = 1
    (2, [0, 8], 0, 0),                 # empty lattice
    (2, [8, 8], 0, 1),                 # FP64 compute with FP32 storage
    (2, [8, 8], 1, 0),                 # FP32 compute with FP64 storage
    (2, [8, 8], 2, 2),                 # FP16 compute
])
def test_required_bytes_rejects(lib, lat, dims, comp, stor):
    o = lbm.lbm_default_opts()
    o.compute, o.storage = comp, stor
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_required_bytes(lat, dims, o)
    assert e.value.code == lbm.LBM_ERR_ARG


def _create_code(lib, lat, dims, nu, bc, opts=None):
    h = ctypes.c_void_p()
    d = np.asarray(dims, dtype=np.int64)
    code = lib.lbm_create(ctypes.byref(h), lat, d.ctypes.data_as(ctypes.c_void_p), nu, bc, 0.1,
                          ctypes.byref(opts) if opts is not None else None)
    if h:
        lib.lbm_destroy(h)
    return code


@pytest.mark.parametrize("lat,dims,nu,bc", [
    (2, [16, 16], 0.0, 0),     # nu must be > 0 (tau > 1/2, Eq. visco-tau)
    (2, [16, 16], -1e-3, 0),
    (2, [16, 16], float("nan"), 0),
    (1, [16, 1], 1e-3, 2),     # cavity is D2Q9 only
    (2, [2, 16], 1e-3, 2),     # cavity needs 3 x 3 nodes
    (2, [16, 16], 1e-3, 7),    # bad boundary kind
])
def test_create_rejects_bad_arguments(lib, lat, dims, nu, bc):
    assert _create_code(lib, lat, dims, nu, bc) == lbm.LBM_ERR_ARG


def test_null_handles_are_rejected(lib):
    assert lib.lbm_step(None, 1) == lbm.LBM_ERR_ARG
    assert lib.lbm_init(None, None, None, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_moments(None, None, None, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_conservation(None, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_stream_function(None, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_stream_function_device(None, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_destroy(None) == lbm.LBM_OK


def test_create_without_device_reports_nodev(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a CUDA device is present")
    except ImportError:
        pass
    assert _create_code(lib, 2, [16, 16], 1e-3, 0) == lbm.LBM_ERR_NODEV


def _header_enum(name):
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef enum\s*\{([^}]*)\}\s*" + name + r"\s*;", src).group(1)
    return {k: int(v) for k, v in re.findall(r"(LBM_[A-Z0-9_]+)\s*=\s*(-?\d+)", body)}


def test_enums_match_header(lib):
    coll = _header_enum("lbm_collision")
    assert coll == {"LBM_MINXENT4": lbm.LBM_MINXENT4, "LBM_SRT": lbm.LBM_SRT,
                    "LBM_MINXENT2": lbm.LBM_MINXENT2, "LBM_MRT": lbm.LBM_MRT,
                    "LBM_TRT": lbm.LBM_TRT}
    assert set(lbm.COLLISIONS.values()) == set(coll.values())
    t2 = _header_enum("lbm_tau2_reading")
    assert t2 == {"LBM_TAU2_PRINTED": lbm.LBM_TAU2_PRINTED, "LBM_TAU2_MAGIC": lbm.LBM_TAU2_MAGIC}
    assert set(lbm.TAU2_READINGS.values()) == set(t2.values())


def test_opts_struct_size_matches(lib):
    """lbm_default_opts clears sizeof(lbm_opts) bytes: a sentinel just past
    the binding's struct must survive (the binding's layout is not shorter
    than the library's), and the defaults land in the binding's fields."""
    n = ctypes.sizeof(lbm.lbm_opts)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xAB] * (n + 64)))
    lib.lbm_default_opts(ctypes.cast(buf, ctypes.POINTER(lbm.lbm_opts)))
    assert all(b == 0xAB for b in bytes(buf)[n:])
    o = lbm.lbm_opts.from_buffer_copy(bytes(buf)[:n])
    assert (o.collision, o.tau2_reading, o.reserved, o.autotune) == (0, 0, 0, 1)


@pytest.mark.parametrize("field,value", [("collision", 5), ("collision", -1),
                                         ("tau2_reading", 2), ("reserved", 1)])
def test_required_bytes_rejects_bad_options(lib, field, value):
    o = lbm.lbm_default_opts()
    setattr(o, field, value)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_required_bytes(lbm.LBM_D2Q9, [8, 8], o)
    assert e.value.code == lbm.LBM_ERR_ARG


@pytest.mark.parametrize("coll", [0, 1, 2, 3, 4])
def test_every_collision_is_accepted(lib, coll):
    o = lbm.lbm_default_opts()
    o.collision = coll
    o.tau2_reading = lbm.LBM_TAU2_MAGIC
    assert lbm.lbm_required_bytes(lbm.LBM_D2Q9, [8, 8], o) > 0
