"""Pins of the oracle's DFT conventions, spectral operators and CIC
assignment: closed forms, invariants and brute force on tiny meshes."""
import itertools

import numpy as np
import pytest

from oracle import mesh as M


def test_dft_convention_delta_and_parseval():
    n = 8
    f = np.zeros((n, n, n))
    f[0, 0, 0] = 1.0
    fk = M.rfft3(f)
    np.testing.assert_allclose(fk, np.ones_like(fk), atol=1e-15)   # X(k) = sum x e^{-ikx}
    rng = np.random.default_rng(0)
    g = rng.standard_normal((n, n, n))
    gk = M.rfft3(g)
    w = np.full(n // 2 + 1, 2.0)
    w[0] = w[-1] = 1.0
    assert np.isclose(np.sum(g * g), np.sum(w * np.abs(gk) ** 2) / n ** 3, rtol=1e-13)
    np.testing.assert_allclose(M.irfft3(gk, n), g, atol=1e-14)


def test_derivative_of_plane_wave():
    n, box = 16, 40.0
    x = np.arange(n) * box / n
    k0 = 2 * np.pi / box * 3
    f = np.broadcast_to(np.cos(k0 * x)[None, :, None], (n, n, n)).copy()   # varies along y
    for ax in range(3):
        d = M.apply_multiplier(f, M.deriv(n, box, ax))
        expect = -k0 * np.sin(k0 * x)[None, :, None] if ax == 1 else 0.0
        np.testing.assert_allclose(d, np.broadcast_to(expect, (n, n, n)), atol=1e-12)
    # inverse Laplacian: lap^{-1} cos = -cos / k0^2
    phi = M.apply_multiplier(f, -M.inv_k2(n, box))
    np.testing.assert_allclose(phi, -f / k0 ** 2, atol=1e-13)


def test_derivative_zero_at_nyquist_and_hermitian():
    n, box = 8, 10.0
    d0 = M.deriv(n, box, 0)
    assert np.all(d0[n // 2] == 0)
    dz = M.deriv(n, box, 2)
    assert np.all(dz[:, :, n // 2] == 0)
    # applying a derivative to any real field gives a real field whose
    # transpose is minus itself: <D f, g> = -<f, D g>
    rng = np.random.default_rng(1)
    f, g = rng.standard_normal((2, n, n, n))
    for ax in range(3):
        a = np.sum(M.apply_multiplier(f, M.deriv(n, box, ax)) * g)
        b = np.sum(f * M.apply_multiplier(g, M.deriv(n, box, ax)))
        assert abs(a + b) < 1e-12


def _brute_paint(u, n, w):
    out = np.zeros((n, n, n))
    for p in range(u.shape[0]):
        for c in itertools.product(range(n), repeat=3):
            wt = 1.0
            for d in range(3):
                # periodic distance to node c_d, nearest image
                dist = (u[p, d] - c[d]) % n
                dist = min(dist, n - dist)
                wt *= max(0.0, 1.0 - dist)
            out[c] += w[p] * wt
    return out


def test_cic_paint_matches_brute_force():
    n = 4
    rng = np.random.default_rng(2)
    u = rng.uniform(-6, 10, (5, 3))
    w = rng.standard_normal(5)
    np.testing.assert_allclose(M.cic_paint(u, n, weights=w), _brute_paint(u, n, w), atol=1e-13)


def test_cic_mass_conservation_and_lattice():
    n = 16
    rng = np.random.default_rng(3)
    u = M.lattice_cells(n) + rng.normal(0, 2.0, (n ** 3, 3))
    rho = M.cic_paint(u, n)
    assert abs(rho.sum() - n ** 3) < 1e-9
    # unperturbed lattice on the nodes paints exactly one per node
    np.testing.assert_array_equal(M.cic_paint(M.lattice_cells(n), n), np.ones((n, n, n)))
    # a uniform sub-cell shift of the whole lattice still paints one per node
    shifted = M.lattice_cells(n) + np.array([0.3, 0.65, 0.1])
    np.testing.assert_allclose(M.cic_paint(shifted, n), np.ones((n, n, n)), atol=1e-14)


def test_paint_readout_adjoint():
    n = 12
    rng = np.random.default_rng(4)
    u = M.lattice_cells(n) + rng.normal(0, 1.5, (n ** 3, 3))
    w = rng.standard_normal(n ** 3)
    m = rng.standard_normal((n, n, n))
    lhs = np.sum(M.cic_paint(u, n, weights=w) * m)
    rhs = np.sum(w * M.cic_readout(u, m))
    assert abs(lhs - rhs) < 1e-12 * np.sqrt(n ** 3) * 10


def test_readout_gradient_matches_finite_difference():
    n = 8
    rng = np.random.default_rng(5)
    u = rng.uniform(0, n, (40, 3))
    m = rng.standard_normal((n, n, n))
    g = M.cic_readout_grad(u, m)
    eps = 1e-6
    for d in range(3):
        up, um = u.copy(), u.copy()
        up[:, d] += eps
        um[:, d] -= eps
        fd = (M.cic_readout(up, m) - M.cic_readout(um, m)) / (2 * eps)
        # away from cell faces the readout is smooth
        frac = u[:, d] - np.floor(u[:, d])
        ok = (frac > 1e-4) & (frac < 1 - 1e-4)
        np.testing.assert_allclose(g[ok, d], fd[ok], atol=1e-8)


def test_readout_gradient_floor_convention_on_a_face():
    # exactly on a node the particle belongs to the cell above it
    n = 4
    m = np.zeros((n, n, n))
    m[1, 0, 0], m[2, 0, 0], m[0, 0, 0] = 1.0, 5.0, -3.0
    u = np.array([[1.0, 0.0, 0.0]])
    g = M.cic_readout_grad(u, m)
    assert g[0, 0] == pytest.approx(m[2, 0, 0] - m[1, 0, 0])
