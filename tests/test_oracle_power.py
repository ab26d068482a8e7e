"""Pins of the power-spectrum estimator: white noise has P = Delta^3, a single
mode lands in its own bin with the closed-form amplitude, r_c(a, a) = 1."""
import numpy as np

from oracle import power
from paper_2604_26823_gb300 import inputs


def test_white_noise_power_is_cell_volume():
    n, box = 32, 64.0
    s = inputs.white_noise(n, 1).astype(np.float64)
    edges = np.linspace(0.2, np.pi * n / box, 8)
    _, pk, nm = power.power_spectrum(s, box, edges)
    assert np.all(np.abs(pk / (box / n) ** 3 - 1) < 6 * np.sqrt(1.0 / nm) + 0.02)


def test_single_mode_amplitude_and_self_correlation():
    n, box = 16, 50.0
    x = np.arange(n) * box / n
    k0 = 2 * np.pi / box * 3
    a = 0.5 * np.cos(k0 * x)[:, None, None] * np.ones((1, n, n))
    edges = np.array([k0 * 0.99, k0 * 1.01])
    k, pk, nm = power.power_spectrum(a, box, edges)
    # two modes (+k0, -k0) with |delta(k)|^2 = (0.5 n^3 / 2)^2 each, P = V |delta|^2 / N^6
    # |n|^2 = 9: (+-3,0,0) and permutations (6) plus (+-2,+-2,+-1) and permutations (24);
    # only the x pair carries power
    assert nm[0] == 30.0
    assert np.isclose(pk[0] * nm[0], 2 * box ** 3 * (0.25 * n ** 3) ** 2 / n ** 6)
    _, r, _ = power.cross_correlation(a + 0.01 * inputs.white_noise(n, 2), a + 0.01 * inputs.white_noise(n, 2), box, edges)
    assert np.isclose(r[0], 1.0)
