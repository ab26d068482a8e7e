"""Analysis utilities on the GPU (Sec. 3.2 r_c(k), Sec. 3.3 T-web) against the
oracle.

Tolerances: mode counts per bin are bit-exact (both sides form the bin index
with the same FP64 expression); binned powers agree to FP32 FFT rounding
(1e-5 relative) or FP64 rounding (1e-11); smoothing 1e-5 / 1e-12 relative L2.
T-web: eigenvalues within 1e-5 (FP32) / 1e-10 (FP64) of the largest |lambda|;
a label is a floating-point decision, so labels must agree wherever every
eigenvalue is farther than that tolerance from lambda_th (elsewhere they must
lie between the counts at lambda_th -+ tolerance); eigenvectors are unique up
to sign only where their eigenvalue is separated from the others, so
|cos| > 1 - 1e-6 is required where the gap exceeds 1e-2 (FP32) / 1e-6 (FP64)
of the largest |lambda|."""
import numpy as np
import pytest

from oracle import analysis as OA
from gpu_cases import rel_l2, table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2604_26823_gb300 import build
    build.build()
    from paper_2604_26823_gb300 import api as A
    return A


def _dt(prec):
    return torch.float32 if prec == "f32" else torch.float64


def _dev(x, prec):
    return torch.tensor(np.ascontiguousarray(x), dtype=_dt(prec), device="cuda")


def _plan(api, n, prec, box):
    lnk, lnp = table()
    return api.Plan(api.Config(n=n, box=box, n_steps=2, precision=prec), lnk, lnp)


def _field(n, seed, scale=1.0):
    from paper_2604_26823_gb300 import inputs
    return inputs.normal_field(n, seed, scale).astype(np.float64)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n", [16, 32, 64])
def test_power_spectra_match_oracle(api, n, prec):
    box = 100.0
    a = _field(n, 41)
    b = (0.6 * a + 0.8 * _field(n, 42)).astype(np.float32).astype(np.float64)
    plan = _plan(api, n, prec, box)
    kf = 2 * np.pi / box
    nb, kmin, kmax = 12, 0.5 * kf, kf * n / 2
    _, paa, pbb, pab, cnt, r = api.pm_power_spectra(plan, _dev(a, prec), _dev(b, prec), nb, kmin, kmax)
    raa, rbb, rab, rcnt = OA.power_spectra(a, b, box, nb, kmin, kmax)
    np.testing.assert_array_equal(cnt, rcnt)
    tol = 1e-5 if prec == "f32" else 1e-11
    ok = rcnt > 0
    for got, ref in ((paa, raa), (pbb, rbb), (pab, rab)):
        np.testing.assert_allclose(got[ok], ref[ok], rtol=tol, atol=tol * np.abs(raa[ok]).max())
    np.testing.assert_allclose(r[ok], OA.correlation_coefficient(raa, rbb, rab)[ok], atol=10 * tol)
    _, paa1, pbb1, pab1, cnt1, _ = api.pm_power_spectra(plan, _dev(a, prec), None, nb, kmin, kmax)
    np.testing.assert_array_equal(cnt1, rcnt)
    np.testing.assert_allclose(paa1[ok], raa[ok], rtol=tol)
    assert np.all(pbb1[ok] == 0) and np.all(pab1[ok] == 0)
    plan.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_smooth_matches_oracle(api, prec):
    n, box = 32, 64.0
    x = _field(n, 43)
    plan = _plan(api, n, prec, box)
    for r_sm in (0.0, 2.0, 5.5):
        got = api.pm_smooth(plan, _dev(x, prec), r_sm).cpu().numpy()
        assert rel_l2(got, OA.smooth(x, box, r_sm)) < (1e-5 if prec == "f32" else 1e-12)
    plan.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n", [16, 32])
def test_tweb_matches_oracle(api, n, prec):
    box, r_sm, th = 2.0 * n, 2.0, 0.16
    delta = _field(n, 44, 0.8)
    plan = _plan(api, n, prec, box)
    labels, eig, evec = api.pm_tweb(plan, _dev(delta, prec), r_sm, th)
    rl, rlam, rvec = OA.tweb(delta, box, r_sm, th)
    lam = eig.cpu().numpy().reshape(3, -1).T.astype(np.float64)
    vec = evec.cpu().numpy().reshape(3, 3, -1).transpose(2, 1, 0).astype(np.float64)   # [cell, comp, which]
    labels = labels.cpu().numpy().reshape(-1)
    scale = np.abs(rlam).max()
    tol = (1e-5 if prec == "f32" else 1e-10) * scale
    assert np.abs(lam - rlam).max() < tol
    lo = np.sum(rlam > th + tol, axis=1)
    hi = np.sum(rlam > th - tol, axis=1)
    assert np.all((labels >= lo) & (labels <= hi))
    clear = lo == hi
    assert clear.mean() > 0.99
    np.testing.assert_array_equal(labels[clear], rl[clear])
    gap_min = (1e-2 if prec == "f32" else 1e-6) * scale
    for i in range(3):
        others = [j for j in range(3) if j != i]
        gap = np.min(np.abs(rlam[:, [i]] - rlam[:, others]), axis=1)
        sep = gap > gap_min
        assert sep.mean() > 0.9
        cos = np.abs(np.sum(vec[:, :, i] * rvec[:, :, i], axis=1))
        assert np.all(cos[sep] > 1 - 1e-6), (i, cos[sep].min())
    # the eigenvectors form an orthonormal frame in every cell
    gram = np.einsum("cki,ckj->cij", vec, vec)
    assert np.abs(gram - np.eye(3)).max() < (1e-5 if prec == "f32" else 1e-12)
    # cosine kernel against the oracle's formula on the same two fields
    rv_dev = _dev(rvec.transpose(2, 1, 0).reshape(3, 3, n, n, n), prec)
    cos_gpu = api.pm_eigvec_cosines(evec, rv_dev).cpu().numpy().reshape(3, -1).T
    np.testing.assert_allclose(cos_gpu, OA.eigvec_cosines(vec, rvec), atol=1e-6 if prec == "f32" else 1e-12)
    plan.close()


def test_confusion_matches_oracle(api):
    rng = np.random.default_rng(45)
    n3 = 40000
    t = rng.integers(0, 4, n3).astype(np.int32)
    r = rng.integers(0, 4, n3).astype(np.int32)
    R = (rng.random(n3) < 0.55) * rng.random(n3)
    got = api.pm_confusion(torch.tensor(t, device="cuda"), torch.tensor(r, device="cuda"),
                           torch.tensor(R, dtype=torch.float32, device="cuda"))
    np.testing.assert_array_equal(got, OA.confusion(t, r, R > 0))
    got_all = api.pm_confusion(torch.tensor(t, device="cuda"), torch.tensor(r, device="cuda"))
    np.testing.assert_array_equal(got_all, OA.confusion(t, r, np.ones(n3, bool)))
