"""Host-side helpers of the cavity studies (no GPU): vortex extrema and the
stability-map reduction."""
import numpy as np

from paper_1801_03863_gb300 import cavity


def test_vortex_centres_on_a_synthetic_field():
    n = 33
    y, x = np.mgrid[0:n, 0:n] / (n - 1)
    psi = -np.exp(-((x - 0.55) ** 2 + (y - 0.6) ** 2) / 0.02)
    psi += 0.01 * np.exp(-((x - 0.85) ** 2 + (y - 0.1) ** 2) / 0.002)
    psi += 0.002 * np.exp(-((x - 0.1) ** 2 + (y - 0.1) ** 2) / 0.002)
    c = cavity.vortex_centres(psi)
    assert c["main"][3:] == (round(0.55 * 32), round(0.6 * 32))
    assert c["lower_right"][3:] == (round(0.85 * 32), round(0.1 * 32))
    assert c["lower_left"][3:] == (round(0.1 * 32), round(0.1 * 32))
    assert c["main"][0] < 0 < c["lower_left"][0] < c["lower_right"][0]


def test_normalisation_and_viscosity():
    psi = np.ones((5, 9))
    assert np.allclose(cavity.normalised_stream_function(psi, 0.1), 1.0 / (0.1 * 8))
    # Eq. (visco-tau): tau = 3 nu + 1/2
    for t in (1.0, 1.5, 1.99):
        assert abs(3 * cavity.nu_from_inv_tau(t) + 0.5 - 1.0 / t) < 1e-15


def test_max_stable_lid_reads_the_first_failure():
    m = cavity.StabilityMap(np.array([1.0, 1.9]), np.array([0.1, 0.2, 0.3]),
                            np.array([[True, True, False], [False, True, True]]),
                            np.zeros((2, 3), int))
    assert list(m.max_stable_lid()) == [0.2, 0.0]
