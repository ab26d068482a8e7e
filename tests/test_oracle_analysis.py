"""Pins of the analysis oracle (power spectra, r_c, smoothing, T-web,
eigenvector cosines, confusion matrix) against closed forms, Parseval's
identity, the trace identity of the deformation tensor and brute force."""
import numpy as np
import pytest

from oracle import analysis as OA
from paper_2604_26823_gb300 import inputs


def _x(n):
    return np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")


def _wave(n, m, amp=1.0):
    x = _x(n)
    return amp * np.cos(2 * np.pi * sum(mi * xi for mi, xi in zip(m, x)) / n)


def test_white_noise_power_is_cell_volume():
    n, box = 32, 100.0
    s = inputs.white_noise(n, 31).astype(np.float64)
    kf = 2 * np.pi / box
    paa, _, _, cnt = OA.power_spectra(s, None, box, 8, kf, kf * n / 2)
    mean = np.sum(paa * cnt) / np.sum(cnt)
    assert mean == pytest.approx((box / n) ** 3, rel=5 / np.sqrt(cnt.sum()))


def test_plane_wave_power_closed_form():
    n, box, m, amp = 16, 50.0, (2, -1, 3), 0.7
    a = _wave(n, m, amp)
    kf = 2 * np.pi / box
    nb, kmin, kmax = 10, 0.5 * kf, kf * 8.5
    paa, _, _, cnt = OA.power_spectra(a, None, box, nb, kmin, kmax)
    b = int(np.floor((kf * np.sqrt(sum(mi * mi for mi in m)) - kmin) / ((kmax - kmin) / nb)))
    expect = np.zeros(nb)
    expect[b] = box ** 3 * amp ** 2 / 2 / cnt[b]
    np.testing.assert_allclose(paa, expect, rtol=1e-12, atol=1e-12 * expect[b])


def test_parseval_over_all_modes():
    n, box = 16, 40.0
    a = inputs.normal_field(n, 32).astype(np.float64)
    kf = 2 * np.pi / box
    paa, _, _, cnt = OA.power_spectra(a, None, box, 5, 0.0, kf * n)       # every mode, k = 0 included
    assert cnt.sum() == n ** 3
    assert np.sum(paa * cnt) == pytest.approx(box ** 3 / n ** 3 * np.sum(a * a), rel=1e-12)


def test_correlation_coefficient_limits():
    n, box = 16, 40.0
    a = inputs.normal_field(n, 33).astype(np.float64)
    c = inputs.normal_field(n, 34).astype(np.float64)
    kf = 2 * np.pi / box
    args = (box, 6, kf, kf * 8)
    np.testing.assert_allclose(OA.correlation_coefficient(*OA.power_spectra(a, 2.5 * a, *args)[:3]), 1.0, rtol=1e-12)
    np.testing.assert_allclose(OA.correlation_coefficient(*OA.power_spectra(a, -a, *args)[:3]), -1.0, rtol=1e-12)
    paa, pbb, pab, cnt = OA.power_spectra(a, c, *args)
    r = OA.correlation_coefficient(paa, pbb, pab)
    assert np.all(np.abs(r) < 6 / np.sqrt(cnt))                            # independent fields


def test_smoothing_closed_form():
    n, box, m, r_sm = 16, 64.0, (1, 2, 0), 3.0
    a = _wave(n, m) + 0.25
    k2 = (2 * np.pi / box) ** 2 * sum(mi * mi for mi in m)
    np.testing.assert_allclose(OA.smooth(a, box, r_sm), _wave(n, m) * np.exp(-0.5 * k2 * r_sm ** 2) + 0.25,
                               atol=1e-12)
    np.testing.assert_allclose(OA.smooth(a, box, 0.0), a, atol=1e-12)


def test_tweb_plane_wave():
    """delta = A cos(k.x): psi = khat khat^T G delta, eigenvalues {0, 0, G delta},
    label 1 where G delta > lambda_th, else 0; the eigenvector of the nonzero
    eigenvalue is +-khat."""
    n, box, m, amp, r_sm, th = 16, 32.0, (1, 2, 2), 1.3, 1.0, 0.16
    d = _wave(n, m, amp)
    kf = 2 * np.pi / box
    g = np.exp(-0.5 * kf * kf * 9 * r_sm ** 2)
    ds = (g * d).ravel()
    labels, lam, vec = OA.tweb(d, box, r_sm, th)
    ref = np.sort(np.stack([ds, np.zeros_like(ds), np.zeros_like(ds)], axis=1), axis=1)
    np.testing.assert_allclose(lam, ref, atol=1e-12)
    np.testing.assert_array_equal(labels, (ds > th).astype(int))
    khat = np.array(m, float) / 3.0
    big = np.abs(ds) > 1e-3
    pos = ds > 0
    col = np.where(pos, 2, 0)
    e = vec[np.arange(ds.size), :, col]
    np.testing.assert_allclose(np.abs(e[big] @ khat), 1.0, atol=1e-9)


def test_tweb_axis_waves_diagonal():
    """Three axis-aligned waves: psi is diagonal with entries G_a A_a cos(.);
    the eigenvalues are those entries sorted and the label counts them above
    lambda_th."""
    n, box, r_sm, th = 16, 32.0, 0.7, 0.16
    x = _x(n)
    amps, ms = (0.9, -0.6, 0.4), (1, 3, 2)
    kf = 2 * np.pi / box
    terms = [a * np.exp(-0.5 * (kf * m) ** 2 * r_sm ** 2) * np.cos(2 * np.pi * m * xi / n)
             for a, m, xi in zip(amps, ms, x)]
    d = sum(a * np.cos(2 * np.pi * m * xi / n) for a, m, xi in zip(amps, ms, x))
    labels, lam, _ = OA.tweb(d, box, r_sm, th)
    w = np.stack([t.ravel() for t in terms], axis=1)
    np.testing.assert_allclose(lam, np.sort(w, axis=1), atol=1e-12)
    np.testing.assert_array_equal(labels, np.sum(w > th, axis=1))


def test_deformation_trace_is_smoothed_density():
    """sum_i psi_ii = G delta minus its mean, for a field without Nyquist-plane modes."""
    n, box, r_sm = 16, 40.0, 2.0
    X = np.fft.fftn(inputs.normal_field(n, 35).astype(np.float64))
    X[n // 2], X[:, n // 2], X[:, :, n // 2] = 0, 0, 0
    d = np.fft.ifftn(X).real + 0.3
    p = OA.deformation_tensor(d, box, r_sm)
    sm = OA.smooth(d, box, r_sm)
    np.testing.assert_allclose(p[0] + p[1] + p[2], sm - sm.mean(), atol=1e-12)


def test_eigvec_cosines():
    rng = np.random.default_rng(36)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    va = np.broadcast_to(q, (5, 3, 3)).copy()
    vb = va.copy()
    vb[:, :, 1] *= -1.0                                       # a sign flip changes nothing
    np.testing.assert_allclose(OA.eigvec_cosines(va, vb), 1.0, atol=1e-14)
    vc = va[:, :, [1, 0, 2]]                                  # swapped e1, e2: orthogonal
    np.testing.assert_allclose(OA.eigvec_cosines(va, vc), [0.0, 0.0, 1.0] * np.ones((5, 1)), atol=1e-14)


def test_confusion_brute_force():
    rng = np.random.default_rng(37)
    t = rng.integers(0, 4, 500)
    r = rng.integers(0, 4, 500)
    mask = rng.random(500) < 0.6
    ref = np.zeros((4, 4), int)
    for i in range(500):
        if mask[i]:
            ref[t[i], r[i]] += 1
    np.testing.assert_array_equal(OA.confusion(t, r, mask), ref)
