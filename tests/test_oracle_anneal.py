"""Pins of the annealing oracle (resolution transfer of the white noise and
coarsening of the data) against closed forms, brute-force DFT sums and
brute-force block sums."""
import numpy as np
import pytest

from oracle import anneal as A
from paper_2604_26823_gb300 import inputs


def _grid(n):
    return np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")


def _no_nyquist(s):
    """s with every mode on a Nyquist plane removed (n even)."""
    n = s.shape[0]
    S = np.fft.fftn(s)
    S[n // 2, :, :] = 0
    S[:, n // 2, :] = 0
    S[:, :, n // 2] = 0
    return np.fft.ifftn(S).real


@pytest.mark.parametrize("nc,n,m", [(8, 16, (1, -2, 3)), (4, 16, (0, 1, -1)), (8, 32, (3, 0, 2))])
def test_plane_wave_closed_form(nc, n, m):
    """A resolved coarse plane wave cos(2 pi m.y / n_c) becomes the same wave
    on the fine mesh, cos(2 pi m.x / n), times r^{-3/2}: the linear density
    s sqrt(P / Delta^3) of the wave is unchanged, since Delta^{-3/2} grows by
    r^{3/2}."""
    r = n // nc
    y = _grid(nc)
    x = _grid(n)
    sc = np.cos(2 * np.pi * sum(mi * yi for mi, yi in zip(m, y)) / nc)
    out = A.refine_noise(sc, np.zeros((n, n, n)))
    ref = r ** -1.5 * np.cos(2 * np.pi * sum(mi * xi for mi, xi in zip(m, x)) / n)
    np.testing.assert_allclose(out, ref, atol=1e-12)


@pytest.mark.parametrize("nc,n", [(8, 16), (4, 16), (16, 32)])
def test_interpolates_through_the_coarse_samples(nc, n):
    """With no fresh noise and no coarse Nyquist content, the fine field is the
    band-limited interpolant: at the coarse nodes it equals r^{-3/2} s_c."""
    r = n // nc
    sc = _no_nyquist(inputs.white_noise(nc, 11).astype(np.float64))
    out = A.refine_noise(sc, np.zeros((n, n, n)))
    np.testing.assert_allclose(out[::r, ::r, ::r], sc / r ** 1.5, atol=1e-12)


def test_fresh_modes_by_brute_force_dft():
    """With s_c = 0 the fine field has no mode inside the coarse cube and
    equals the fresh field's DFT outside it (explicit DFT sums)."""
    nc, n = 4, 8
    fresh = inputs.white_noise(n, 12).astype(np.float64)
    out = A.refine_noise(np.zeros((nc, nc, nc)), fresh)
    x = _grid(n)

    def dft(f, k):
        ph = np.exp(-2j * np.pi * sum(ki * xi for ki, xi in zip(k, x)) / n)
        return np.sum(f * ph)

    for k in [(0, 0, 0), (1, -1, 0), (1, 1, 1), (-1, 0, 1)]:        # every |k_i| < nc / 2
        assert abs(dft(out, k)) < 1e-10
    for k in [(2, 0, 0), (0, 3, -1), (4, 4, 4), (1, 2, -3), (-2, 1, 1)]:
        assert abs(dft(out, k) - dft(fresh, k)) < 1e-10


def test_unit_white_noise_is_kept():
    """Coarse and fresh N(0,1) fields give an N(0,1) fine field (variance
    within a few standard errors, mean ~0)."""
    nc, n = 16, 32
    out = A.refine_noise(inputs.white_noise(nc, 13).astype(np.float64),
                         inputs.white_noise(n, 14).astype(np.float64))
    assert abs(out.var() - 1.0) < 5 * np.sqrt(2.0 / n ** 3)
    assert abs(out.mean()) < 5 / np.sqrt(n ** 3)


@pytest.mark.parametrize("n,f", [(4, 2), (8, 4), (8, 2)])
def test_coarsen_by_brute_force(n, f):
    x = inputs.uniform_field(n, 15, 0.0, 3.0).astype(np.float64)
    nc = n // f
    ref = np.zeros((nc, nc, nc))
    for i in range(n):
        for j in range(n):
            for l in range(n):
                ref[i // f, j // f, l // f] += x[i, j, l]
    np.testing.assert_allclose(A.coarsen(x, f), ref, rtol=1e-14)
    np.testing.assert_allclose(A.coarsen(x, f, mean=True), ref / f ** 3, rtol=1e-14)
    assert A.coarsen(x, f).sum() == pytest.approx(x.sum(), rel=1e-14)
