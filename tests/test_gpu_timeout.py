"""The bounded-wait failure path of the TMA-staged step kernel.

Every mbarrier wait of the kernel gives up after a bounded number of polls;
the CTA then sets the context's error word, waits (bounded) for its own
copies still in flight and leaves, and lbm_status / lbm_moments report
LBM_ERR_TIMEOUT.  The test makes one wait run out on purpose without any GPU
fault: the host-side hook LBM_TEST_LOST_TILE makes the producing thread skip
the copies of one tile, so that tile's full barrier never completes (nothing
is in flight for it), and LBM_SPIN_LIMIT shortens the waits (65536 polls,
still far longer than any real copy takes).  A context created afterwards on
the same device runs normally.
"""
import numpy as np
import pytest

from paper_1801_03863_gb300 import lbm

pytestmark = pytest.mark.gpu


def _cavity(nx, ny):
    return np.full(nx * ny, 1.0), np.zeros(nx * ny), np.zeros(nx * ny)


@pytest.mark.parametrize("shape,lost", [("smem", 5), ("smem", 0), ("smems", 3), ("smemw", 4),
                                               ("smemd", 6)])
def test_lost_copy_times_out_and_is_reported(shape, lost, monkeypatch):
    nx, ny = 256, 64  # 10 large tiles, 20 small ones, 8 of the 10-warp CTAs', 10 deep-ring ones
    monkeypatch.setenv("LBM_SHAPE", shape)
    monkeypatch.setenv("LBM_SPIN_LIMIT", "65536")
    monkeypatch.setenv("LBM_TEST_LOST_TILE", str(lost))
    fields = _cavity(nx, ny)
    with lbm.Lattice("d2q9", [(nx, ny)], 0.02, "cavity", u_lid=0.05, compute="f32",
                     storage="f16") as lat:
        lat.init(*fields)
        lat.step(3)  # the in-place first collision, then two TMA-kernel steps
        lat.stream.synchronize()
        with pytest.raises(lbm.LBMError) as e:
            lat.status()
        assert e.value.code == lbm.LBM_ERR_TIMEOUT
        with pytest.raises(lbm.LBMError) as e:
            lat.moments()
        assert e.value.code == lbm.LBM_ERR_TIMEOUT
    # the device and a new context are unaffected
    monkeypatch.delenv("LBM_TEST_LOST_TILE")
    monkeypatch.delenv("LBM_SPIN_LIMIT")
    with lbm.Lattice("d2q9", [(nx, ny)], 0.02, "cavity", u_lid=0.05, compute="f32",
                     storage="f16") as lat:
        lat.init(*fields)
        lat.step(3)
        r, x, y = lat.moments()
        assert lat.status()["unstable"] == 0
        assert np.all(np.isfinite(r)) and abs(r.mean() - 1.0) < 1e-3
