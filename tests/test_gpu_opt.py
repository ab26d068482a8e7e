"""GPU parity of the projection operator, rank-order matching and the L-BFGS
step against the oracle, through the C ABI.

Integer / index results are compared bit for bit: the real-space matching
permutation (both sides sort the same FP32 values), the number of resets,
the per-bin multiset of the Fourier matching.  Floating-point results use
the FP32 path's 1e-5 relative tolerance (1e-12 on the FP64 path).
"""
import numpy as np
import pytest

from oracle import lbfgs as OL
from oracle import mesh as OMesh
from oracle import projection as OP
from gpu_cases import rel_l2, table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2604_26823_gb300 import build
    build.build()
    from paper_2604_26823_gb300 import api as A
    return A


_PLANS = {}


def plan(api, n, box, prec):
    key = (n, box, prec)
    if key not in _PLANS:
        lnk, lnp = table()
        _PLANS[key] = api.Plan(api.Config(n=n, box=box, precision=prec, n_steps=1), lnk, lnp)
    return _PLANS[key]


def dt(prec):
    return torch.float32 if prec == "f32" else torch.float64


def dev(x, prec):
    return torch.tensor(np.asarray(x), dtype=dt(prec), device="cuda")


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n", [16, 64])
def test_projection_with_resets(api, n, prec):
    from paper_2604_26823_gb300 import inputs
    p = plan(api, n, 100.0, prec)
    s = (3.0 + 2.0 * inputs.white_noise(n, 1)).astype(np.float32)
    s.reshape(-1)[[7, 100, n ** 3 - 1]] = [300.0, -250.0, 280.0]
    x = dev(s, prec)
    nres = api.project_rank_match(p, x, api.L.PM_PROJECT, seed=6, counter=11)
    ref, rn = OP.project(s.astype(np.float64), 6, 11)
    assert nres == rn == 3
    tol = 1e-6 if prec == "f32" else 1e-12
    np.testing.assert_allclose(x.cpu().numpy(), ref, rtol=tol, atol=tol)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n", [16, 64])
def test_real_rom_bit_exact(api, n, prec):
    from paper_2604_26823_gb300 import inputs
    p = plan(api, n, 100.0, prec)
    s = inputs.white_noise(n, 2)
    s.reshape(-1)[5:40] = 0.25       # ties, broken by index
    s.reshape(-1)[50] = -0.0
    s.reshape(-1)[51] = 0.0
    resp = inputs.uniform_field(n, 3, -0.6, 1.0)
    cnt = api.pm_count_positive(p, dev(resp, prec))
    assert cnt == int((resp > 0).sum())
    t = inputs.sorted_normal_targets(cnt, 4)
    x = dev(s, prec)
    api.project_rank_match(p, x, api.L.PM_ROM_REAL, R=dev(resp, prec), targets_real=dev(t, prec))
    ref = OP.rom_real(s.astype(np.float64), resp.astype(np.float64), t.astype(np.float64))
    np.testing.assert_array_equal(x.cpu().numpy().astype(np.float64), ref)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,box", [(16, 20.0), (64, 300.0)])
def test_fourier_rom(api, n, box, prec):
    from paper_2604_26823_gb300 import inputs
    p = plan(api, n, box, prec)
    counts = api.pm_rom_fourier_counts(p)
    np.testing.assert_array_equal(counts, OP.fourier_bin_counts(n, box))
    s = inputs.white_noise(n, 5).astype(np.float64)
    t = inputs.sorted_normal_targets_per_bin(counts, 6)
    x = dev(s, prec)
    api.project_rank_match(p, x, api.L.PM_ROM_FOURIER, targets_fourier=dev(t, prec))
    got = x.cpu().numpy().astype(np.float64)
    ref = OP.rom_fourier(s, box, t.astype(np.float64))
    # matched multisets per bin are the targets exactly
    idx, b, _ = OP.fourier_modes(n, box)
    z = OMesh.rfft3(got).reshape(-1)[idx] * np.sqrt(2.0 / n ** 3)
    vals = np.empty(2 * idx.size)
    vals[0::2], vals[1::2] = z.real, z.imag
    eb = np.repeat(b, 2)
    offs = np.concatenate([[0], np.cumsum(counts)])
    tol = 2e-5 if prec == "f32" else 1e-10
    for bb in range(100):
        np.testing.assert_allclose(np.sort(vals[eb == bb]), np.sort(t[offs[bb]:offs[bb + 1]].astype(np.float64)),
                                   atol=tol * 10)
    # the assignment equals the oracle's except where two input values of a
    # bin are closer than the FFT's rounding (then either order is correct)
    _check_fourier_assignment(s, got, ref, box, 2e-5 if prec == "f32" else 1e-12)


def _fourier_values(x, box):
    n = x.shape[0]
    idx, b, _ = OP.fourier_modes(n, box)
    z = OMesh.rfft3(x).reshape(-1)[idx] * np.sqrt(2.0 / n ** 3)
    v = np.empty(2 * idx.size)
    v[0::2], v[1::2] = z.real, z.imag
    return v, np.repeat(b, 2)


def _check_fourier_assignment(s, got, ref, box, tol):
    """Element by element, the matched Fourier values equal the oracle's; an
    element that differs must have swapped targets with one whose input value
    lies within tol of its own (a tie at the FFT's rounding)."""
    vin, eb = _fourier_values(s, box)
    vg, _ = _fourier_values(got, box)
    vr, _ = _fourier_values(ref, box)
    bad = np.nonzero(np.abs(vg - vr) > tol * 10)[0]
    for i in bad:
        # the oracle element that holds the target GPU element i received
        same_bin = np.nonzero(eb == eb[i])[0]
        j = same_bin[np.argmin(np.abs(vr[same_bin] - vg[i]))]
        assert abs(vin[i] - vin[j]) < tol * 10, (i, j, vin[i], vin[j])
    assert bad.size <= max(4, vin.size // 1000), bad.size
    # outside the Fourier matching's modes the field is unchanged up to rounding
    return bad.size


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_composite_mode(api, prec):
    from paper_2604_26823_gb300 import inputs
    n, box = 32, 150.0
    p = plan(api, n, box, prec)
    s = (inputs.white_noise(n, 8) * np.float32(1.7) + np.float32(0.4)).astype(np.float64)
    resp = inputs.uniform_field(n, 9, -1.0, 1.0).astype(np.float64)
    tr = inputs.sorted_normal_targets(int((resp > 0).sum()), 10)
    tf = inputs.sorted_normal_targets_per_bin(OP.fourier_bin_counts(n, box), 11)
    x = dev(s, prec)
    api.project_rank_match(p, x, 7, R=dev(resp, prec), targets_real=dev(tr, prec),
                           targets_fourier=dev(tf, prec), seed=3, counter=4)
    if prec == "f64":
        ref, _ = OP.project_rank_match(s, box, resp, 7,
                                       tr.astype(np.float64), tf.astype(np.float64), seed=3, counter=4)
        assert rel_l2(x.cpu().numpy(), ref) < 1e-10
    # Fourier matching alone, then real matching + projection from its result:
    # the composite call equals the two calls bit for bit, the Fourier stage
    # follows the oracle up to ties at the FFT's rounding, and the second stage
    # follows the oracle run from the GPU's own Fourier result (exact ranks,
    # projection to rounding)
    x1 = dev(s, prec)
    api.project_rank_match(p, x1, api.L.PM_ROM_FOURIER, targets_fourier=dev(tf, prec))
    f1 = x1.cpu().numpy().astype(np.float64)
    _check_fourier_assignment(s, f1, OP.rom_fourier(s, box, tf.astype(np.float64)), box,
                              2e-5 if prec == "f32" else 1e-12)
    api.project_rank_match(p, x1, api.L.PM_ROM_REAL | api.L.PM_PROJECT, R=dev(resp, prec),
                           targets_real=dev(tr, prec), seed=3, counter=4)
    assert torch.equal(x, x1)
    ref2, _ = OP.project_rank_match(f1, box, resp, 5, tr.astype(np.float64), None, seed=3, counter=4)
    assert rel_l2(x1.cpu().numpy(), ref2) < (1e-6 if prec == "f32" else 1e-13)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_lbfgs_matches_oracle(api, prec):
    rng = np.random.default_rng(0)
    n, m = 5000, 4
    a = rng.uniform(0.5, 3.0, n)
    b = rng.standard_normal(n)
    grad = lambda x: a * x - b
    st = api.LBFGS(n, m=m, precision=prec)
    ref = OL.LBFGS(m=m)
    x = np.zeros(n)
    tol = 1e-5 if prec == "f32" else 1e-11
    for it in range(7):
        xq = x.astype(np.float32).astype(np.float64) if prec == "f32" else x
        g = grad(xq)
        gq = g.astype(np.float32).astype(np.float64) if prec == "f32" else g
        d, gd, dn, pushed = api.lbfgs_step(st, dev(xq, prec), dev(gq, prec))
        rd, rgd, rpushed = ref.step(xq, gq)
        assert pushed == rpushed
        assert rel_l2(d.cpu().numpy(), rd) < tol
        assert abs(gd - rgd) < tol * abs(rgd)
        assert abs(dn - np.linalg.norm(rd)) < tol * np.linalg.norm(rd)
        x = xq + 0.5 * d.cpu().numpy().astype(np.float64) / max(1.0, dn)
    api.lbfgs_reset(st)
    d, gd, dn, pushed = api.lbfgs_step(st, dev(x, prec), dev(grad(x), prec))
    assert not pushed
    np.testing.assert_allclose(d.cpu().numpy(), -grad(x), rtol=1e-6)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_axpy(api, prec):
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(1001), rng.standard_normal(1001)
    if prec == "f32":
        x, y = x.astype(np.float32).astype(np.float64), y.astype(np.float32).astype(np.float64)
    out = api.pm_axpy(0.37, dev(x, prec), dev(y, prec))
    # one rounding of the product and one of the sum in the path's precision
    eps = 6e-8 if prec == "f32" else 1.2e-16
    np.testing.assert_allclose(out.cpu().numpy(), y + 0.37 * x, rtol=0, atol=2 * eps * (np.abs(y) + np.abs(0.37 * x)).max())


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_projection_leaves_input_untouched_on_error(api, prec):
    """NaN in s, or zero variance: PM_ERR_NONFINITE, and s keeps its values
    (the projection kernel reads the moments' validity flag on the device)."""
    from paper_2604_26823_gb300 import inputs
    p = plan(api, 16, 100.0, prec)
    s = inputs.white_noise(16, 1)
    s.reshape(-1)[5] = np.nan
    for vec in (s, np.full((16, 16, 16), 2.5, np.float32)):
        x = dev(vec, prec)
        before = x.cpu().numpy().copy()
        with pytest.raises(api.L.PMError) as err:
            api.project_rank_match(p, x, api.L.PM_PROJECT, seed=6, counter=1)
        assert err.value.status == api.L.PM_ERR_NONFINITE
        np.testing.assert_array_equal(x.cpu().numpy(), before)
