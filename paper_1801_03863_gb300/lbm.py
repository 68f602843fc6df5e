"""Python binding of liblbm (include/lbm.h): argument marshalling only.

Every function named ``lbm_*`` here calls the C entry point of the same name;
all lattice arithmetic runs in the library's CUDA kernels.  PyTorch supplies
device memory (the context's block is a torch uint8 tensor passed through
``lbm_opts.device_mem``) and streams.  There is no CPU fallback: if
liblbm.so is missing or no sm_103 GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_ALLOC, LBM_ERR_CUDA = 0, -1, -2, -3
LBM_ERR_UNSTABLE, LBM_ERR_STATE, LBM_ERR_NODEV, LBM_ERR_TIMEOUT = -4, -5, -6, -7
LBM_D1Q3, LBM_D2Q9 = 1, 2
LBM_BC_PERIODIC, LBM_BC_ZERO_GRADIENT, LBM_BC_CAVITY = 0, 1, 2
LBM_MINXENT4, LBM_SRT, LBM_MINXENT2, LBM_MRT, LBM_TRT = 0, 1, 2, 3, 4
LBM_TAU2_PRINTED, LBM_TAU2_MAGIC = 0, 1
LBM_F64, LBM_F32, LBM_F16, LBM_BF16 = 0, 1, 2, 3

DTYPES = {"f64": LBM_F64, "f32": LBM_F32, "f16": LBM_F16, "bf16": LBM_BF16}
COLLISIONS = {"minxent4": LBM_MINXENT4, "srt": LBM_SRT, "minxent2": LBM_MINXENT2, "mrt": LBM_MRT,
              "trt": LBM_TRT}
TAU2_READINGS = {"printed": LBM_TAU2_PRINTED, "magic": LBM_TAU2_MAGIC}
BCS = {"periodic": LBM_BC_PERIODIC, "zero_gradient": LBM_BC_ZERO_GRADIENT, "cavity": LBM_BC_CAVITY}

# Every symbol the header declares (checked by the ABI test).
EXPORTS = (
    "lbm_default_opts", "lbm_required_bytes", "lbm_create", "lbm_create_batch", "lbm_init",
    "lbm_init_device", "lbm_step", "lbm_moments", "lbm_moments_device", "lbm_get_populations",
    "lbm_set_populations", "lbm_conservation", "lbm_conservation_device",
    "lbm_stream_function", "lbm_stream_function_device",
    "lbm_conservation_noalloc", "lbm_status",
    "lbm_status_instance",
    "lbm_launch_shape", "lbm_destroy", "lbm_status_string",
    "lbm_init_batch", "lbm_moments_batch", "lbm_moments_batch_device",
    "lbm_stream_function_batch", "lbm_state_bytes", "lbm_save_state", "lbm_load_state",
)


class lbm_opts(ctypes.Structure):
    _fields_ = [
        ("compute", ctypes.c_int32),
        ("storage", ctypes.c_int32),
        ("collision", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("rho0", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("device_mem", ctypes.c_void_p),
        ("device_mem_bytes", ctypes.c_uint64),
        ("tau2_reading", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class LBMError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {lbm_status_string(code)} ({code})")


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblbm.so (built by ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"liblbm.so not found at {path}: run __graft_entry__.build() first")
        lib = ctypes.CDLL(path)
        P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        OP = ctypes.POINTER(lbm_opts)
        sig = {
            "lbm_default_opts": (None, [OP]),
            "lbm_required_bytes": (ctypes.c_int, [I32, I32, P, OP, ctypes.POINTER(ctypes.c_uint64)]),
            "lbm_create": (ctypes.c_int, [ctypes.POINTER(P), I32, P, D, I32, D, OP]),
            "lbm_create_batch": (ctypes.c_int, [ctypes.POINTER(P), I32, I32, P, P, P, I32, OP]),
            "lbm_init": (ctypes.c_int, [P, P, P, P]),
            "lbm_init_device": (ctypes.c_int, [P, P, P, P]),
            "lbm_step": (ctypes.c_int, [P, I64]),
            "lbm_moments": (ctypes.c_int, [P, P, P, P]),
            "lbm_moments_device": (ctypes.c_int, [P, P, P, P]),
            "lbm_stream_function": (ctypes.c_int, [P, P]),
            "lbm_stream_function_device": (ctypes.c_int, [P, P]),
            "lbm_get_populations": (ctypes.c_int, [P, P]),
            "lbm_set_populations": (ctypes.c_int, [P, P]),
            "lbm_conservation": (ctypes.c_int, [P, P]),
            "lbm_conservation_device": (ctypes.c_int, [P, P]),
            "lbm_conservation_noalloc": (ctypes.c_int, [P, P]),
            "lbm_status": (ctypes.c_int, [P, P]),
            "lbm_status_instance": (ctypes.c_int, [P, I32, P]),
            "lbm_launch_shape": (ctypes.c_int, [P, P]),
            "lbm_destroy": (ctypes.c_int, [P]),
            "lbm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "lbm_init_batch": (ctypes.c_int, [P, I32, P, P, P]),
            "lbm_moments_batch": (ctypes.c_int, [P, I32, P, P, P]),
            "lbm_moments_batch_device": (ctypes.c_int, [P, I32, P, P, P]),
            "lbm_stream_function_batch": (ctypes.c_int, [P, I32, P]),
            "lbm_state_bytes": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_uint64)]),
            "lbm_save_state": (ctypes.c_int, [P, P]),
            "lbm_load_state": (ctypes.c_int, [P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(code: int, where: str, allow_unstable: bool = False) -> int:
    if code == LBM_OK or (allow_unstable and code == LBM_ERR_UNSTABLE):
        return code
    raise LBMError(code, where)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------
# Thin wrappers with the C names.
# ----------------------------------------------------------------------------
def lbm_status_string(code: int) -> str:
    return load().lbm_status_string(int(code)).decode()


def lbm_default_opts() -> lbm_opts:
    o = lbm_opts()
    load().lbm_default_opts(ctypes.byref(o))
    return o


def lbm_required_bytes(lattice: int, dims, opts: lbm_opts) -> int:
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int64).reshape(-1))
    out = ctypes.c_uint64()
    _check(load().lbm_required_bytes(lattice, len(d) // 2, _p(d), ctypes.byref(opts),
                                     ctypes.byref(out)), "lbm_required_bytes")
    return int(out.value)


def lbm_create_batch(lattice: int, dims, nu, u_lid, bc: int, opts: lbm_opts) -> ctypes.c_void_p:
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int64).reshape(-1))
    nu = _f64(nu).reshape(-1)
    ul = None if u_lid is None else _f64(u_lid).reshape(-1)
    h = ctypes.c_void_p()
    _check(load().lbm_create_batch(ctypes.byref(h), lattice, len(d) // 2, _p(d), _p(nu),
                                   None if ul is None else _p(ul), bc, ctypes.byref(opts)),
           "lbm_create_batch")
    return h


def lbm_create(lattice: int, dims, nu: float, bc: int, u_lid: float, opts: lbm_opts):
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int64).reshape(-1))
    h = ctypes.c_void_p()
    _check(load().lbm_create(ctypes.byref(h), lattice, _p(d), float(nu), bc, float(u_lid),
                             ctypes.byref(opts)), "lbm_create")
    return h


def lbm_init(h, rho, ux=None, uy=None) -> None:
    rho = _f64(rho).reshape(-1)
    ux = None if ux is None else _f64(ux).reshape(-1)
    uy = None if uy is None else _f64(uy).reshape(-1)
    _check(load().lbm_init(h, _p(rho), None if ux is None else _p(ux),
                           None if uy is None else _p(uy)), "lbm_init")


def lbm_init_device(h, rho_ptr: int, ux_ptr, uy_ptr) -> None:
    _check(load().lbm_init_device(h, rho_ptr, ux_ptr, uy_ptr), "lbm_init_device")


def lbm_step(h, n: int) -> None:
    _check(load().lbm_step(h, int(n)), "lbm_step")


def lbm_moments(h, n_nodes: int, want_uy: bool = True, allow_unstable: bool = False):
    rho = np.empty(n_nodes)
    ux = np.empty(n_nodes)
    uy = np.empty(n_nodes) if want_uy else None
    code = load().lbm_moments(h, _p(rho), _p(ux), None if uy is None else _p(uy))
    _check(code, "lbm_moments", allow_unstable=allow_unstable)
    return rho, ux, uy, code


def lbm_moments_device(h, rho_ptr: int, ux_ptr, uy_ptr) -> None:
    _check(load().lbm_moments_device(h, rho_ptr, ux_ptr, uy_ptr), "lbm_moments_device")


def lbm_stream_function(h, n_nodes: int, allow_unstable: bool = False) -> np.ndarray:
    psi = np.empty(n_nodes)
    _check(load().lbm_stream_function(h, _p(psi)), "lbm_stream_function",
           allow_unstable=allow_unstable)
    return psi


def lbm_stream_function_device(h, psi_ptr: int) -> None:
    _check(load().lbm_stream_function_device(h, psi_ptr), "lbm_stream_function_device")


def lbm_get_populations(h, n_values: int) -> np.ndarray:
    out = np.empty(n_values)
    _check(load().lbm_get_populations(h, _p(out)), "lbm_get_populations")
    return out


def lbm_set_populations(h, f) -> None:
    f = _f64(f).reshape(-1)
    _check(load().lbm_set_populations(h, _p(f)), "lbm_set_populations")


def lbm_conservation(h, count: int) -> np.ndarray:
    out = np.empty(3 * count)
    _check(load().lbm_conservation(h, _p(out)), "lbm_conservation")
    return out.reshape(count, 3)


def lbm_conservation_device(h, out_ptr) -> None:
    _check(load().lbm_conservation_device(h, out_ptr), "lbm_conservation_device")


def lbm_conservation_noalloc(h, out_ptr) -> None:
    """Conservation totals into device memory without any device allocation
    (scratch in a fixed array inside the library; up to 4096 instances)."""
    _check(load().lbm_conservation_noalloc(h, out_ptr), "lbm_conservation_noalloc")


def lbm_status(h) -> dict:
    c = np.zeros(3, np.int64)
    _check(load().lbm_status(h, _p(c)), "lbm_status")
    return {"newton_skipped": int(c[0]), "unstable": int(c[1]), "steps": int(c[2])}


def lbm_status_instance(h, i: int) -> dict:
    c = np.zeros(3, np.int64)
    _check(load().lbm_status_instance(h, int(i), _p(c)), "lbm_status_instance")
    return {"newton_skipped": int(c[0]), "unstable": int(c[1]), "steps": int(c[2])}


def lbm_launch_shape(h) -> dict:
    c = np.zeros(5, np.int32)
    _check(load().lbm_launch_shape(h, _p(c)), "lbm_launch_shape")
    return {"V": int(c[0]), "tw": int(c[1]), "th": int(c[2]), "grid": int(c[3]),
            "kind": {0: "chunks", 1: "smem", 2: "smem_small", 3: "smem_wide",
                     4: "smem_deep"}[int(c[4])]}


def lbm_init_batch(h, instance: int, rho, ux=None, uy=None) -> None:
    rho = _f64(rho).reshape(-1)
    ux = None if ux is None else _f64(ux).reshape(-1)
    uy = None if uy is None else _f64(uy).reshape(-1)
    _check(load().lbm_init_batch(h, int(instance), _p(rho), None if ux is None else _p(ux),
                                 None if uy is None else _p(uy)), "lbm_init_batch")


def lbm_moments_batch(h, instance: int, n_nodes: int, want_uy: bool = True,
                      allow_unstable: bool = False):
    rho = np.empty(n_nodes)
    ux = np.empty(n_nodes)
    uy = np.empty(n_nodes) if want_uy else None
    code = load().lbm_moments_batch(h, int(instance), _p(rho), _p(ux),
                                    None if uy is None else _p(uy))
    _check(code, "lbm_moments_batch", allow_unstable=allow_unstable)
    return rho, ux, uy, code


def lbm_moments_batch_device(h, instance: int, rho_ptr, ux_ptr, uy_ptr) -> None:
    _check(load().lbm_moments_batch_device(h, int(instance), rho_ptr, ux_ptr, uy_ptr),
           "lbm_moments_batch_device")


def lbm_stream_function_batch(h, instance: int, n_nodes: int,
                              allow_unstable: bool = False) -> np.ndarray:
    psi = np.empty(n_nodes)
    _check(load().lbm_stream_function_batch(h, int(instance), _p(psi)),
           "lbm_stream_function_batch", allow_unstable=allow_unstable)
    return psi


def lbm_state_bytes(h) -> int:
    out = ctypes.c_uint64()
    _check(load().lbm_state_bytes(h, ctypes.byref(out)), "lbm_state_bytes")
    return int(out.value)


def lbm_save_state(h) -> np.ndarray:
    buf = np.empty(lbm_state_bytes(h), dtype=np.uint8)
    _check(load().lbm_save_state(h, _p(buf)), "lbm_save_state")
    return buf


def lbm_load_state(h, buf) -> None:
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(load().lbm_load_state(h, _p(buf)), "lbm_load_state")


def lbm_destroy(h) -> None:
    if h:
        load().lbm_destroy(h)


# ----------------------------------------------------------------------------
# Convenience object: one context whose device block and stream come from torch.
# ----------------------------------------------------------------------------
class Lattice:
    """A context of one or more instances.

    dims: list of (nx, ny); nu, u_lid: per instance.  Device memory is one
    torch uint8 tensor on the current CUDA device; work runs on a dedicated
    torch stream (``self.stream``) unless one is given.
    """

    def __init__(self, lattice: str, dims, nu, bc: str, u_lid=None, compute: str = "f64",
                 storage: str | None = None, collision: str = "minxent4", rho0: float = 1.0,
                 autotune: bool = True, stream=None, torch_memory: bool = True,
                 tau2_reading: str = "printed"):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("liblbm needs a CUDA device (no CPU fallback)")
        load()
        self.lattice = LBM_D2Q9 if lattice.lower() == "d2q9" else LBM_D1Q3
        self.q = 9 if self.lattice == LBM_D2Q9 else 3
        dims = [(int(a), int(b)) for a, b in dims]
        self.dims = dims
        self.count = len(dims)
        self.n_nodes = sum(a * b for a, b in dims)
        nu = np.broadcast_to(np.asarray(nu, dtype=np.float64), (self.count,)).copy()
        ul = None if u_lid is None else np.broadcast_to(
            np.asarray(u_lid, dtype=np.float64), (self.count,)).copy()
        storage = storage or compute
        o = lbm_default_opts()
        o.compute = DTYPES[compute]
        o.storage = DTYPES[storage]
        o.collision = COLLISIONS[collision]
        o.tau2_reading = TAU2_READINGS[tau2_reading]
        o.autotune = int(bool(autotune))
        o.rho0 = float(rho0)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        o.stream = ctypes.c_void_p(self.stream.cuda_stream)
        self._mem = None
        if torch_memory:
            nbytes = lbm_required_bytes(self.lattice, [v for d in dims for v in d], o)
            self._mem = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._mem.data_ptr()
            aligned = (base + 255) // 256 * 256
            o.device_mem = ctypes.c_void_p(aligned)
            o.device_mem_bytes = nbytes
        torch.cuda.synchronize()
        self._h = lbm_create_batch(self.lattice, [v for d in dims for v in d], nu, ul,
                                   BCS[bc], o)
        self.opts = o

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            lbm_destroy(self._h)
            self._h = None
        self._mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state
    def init(self, rho, ux=None, uy=None):
        lbm_init(self._h, rho, ux, uy)

    def init_device(self, rho, ux=None, uy=None):
        """rho/ux/uy: torch float64 CUDA tensors (ordered on self.stream)."""
        ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
        lbm_init_device(self._h, ptr(rho), ptr(ux), ptr(uy))

    def init_instance(self, i: int, rho, ux=None, uy=None):
        """Initial equilibrium of instance i alone (before the first step)."""
        lbm_init_batch(self._h, i, rho, ux, uy)

    def step(self, n: int = 1):
        lbm_step(self._h, n)

    def moments_instance(self, i: int, allow_unstable: bool = False):
        """rho, ux, uy of instance i as [ny, nx] arrays (uy None on D1Q3)."""
        nx, ny = self.dims[i]
        r, x, y, _ = lbm_moments_batch(self._h, i, nx * ny, self.q == 9, allow_unstable)
        return (r.reshape(ny, nx), x.reshape(ny, nx), None if y is None else y.reshape(ny, nx))

    def stream_function_instance(self, i: int, allow_unstable: bool = False) -> np.ndarray:
        nx, ny = self.dims[i]
        return lbm_stream_function_batch(self._h, i, nx * ny, allow_unstable).reshape(ny, nx)

    def save_state(self) -> np.ndarray:
        """Exact checkpoint (raw stored state, step count, counters) as bytes."""
        return lbm_save_state(self._h)

    def load_state(self, buf):
        lbm_load_state(self._h, buf)

    def moments(self, allow_unstable: bool = False):
        rho, ux, uy, _ = lbm_moments(self._h, self.n_nodes, self.q == 9, allow_unstable)
        return rho, ux, uy

    def moments_device(self, rho, ux, uy=None):
        ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
        lbm_moments_device(self._h, ptr(rho), ptr(ux), ptr(uy))

    def stream_function(self, allow_unstable: bool = False) -> np.ndarray:
        """psi of every instance (lattice units), concatenated like moments()."""
        return lbm_stream_function(self._h, self.n_nodes, allow_unstable)

    def stream_function_device(self, psi):
        lbm_stream_function_device(self._h, ctypes.c_void_p(psi.data_ptr()))

    def populations(self) -> np.ndarray:
        return lbm_get_populations(self._h, self.n_nodes * self.q)

    def set_populations(self, f):
        lbm_set_populations(self._h, f)

    def conservation(self) -> np.ndarray:
        return lbm_conservation(self._h, self.count)

    def conservation_device(self, out):
        """out: torch float64 CUDA tensor of 3 * count (ordered on self.stream)."""
        lbm_conservation_device(self._h, ctypes.c_void_p(out.data_ptr()))

    def status(self) -> dict:
        return lbm_status(self._h)

    def status_instance(self, i: int) -> dict:
        return lbm_status_instance(self._h, i)

    def launch_shape(self) -> dict:
        return lbm_launch_shape(self._h)

    def split(self, flat: np.ndarray, per_node: int = 1):
        """Split concatenated per-node arrays into per-instance [ny, nx] arrays."""
        out, k = [], 0
        for nx, ny in self.dims:
            n = nx * ny * per_node
            out.append(flat[k:k + n].reshape((per_node, ny, nx) if per_node > 1 else (ny, nx)))
            k += n
        return out
