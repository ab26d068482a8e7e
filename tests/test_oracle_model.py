"""Pins of the oracle's forward model and adjoint: closed forms (linear
field amplitude, 2LPT of plane waves, single-mode force), invariants
(momentum conservation, unperturbed lattice), the linear-growth limit of
the leapfrog, and brute-force finite differences of the full gradient."""
import numpy as np
import pytest

from oracle import cosmology as C
from oracle import mesh as M
from oracle import model
from oracle import analysis
from paper_2604_26823_gb300 import inputs


@pytest.fixture(scope="module")
def table():
    return C.linear_power_table()


def test_ic_amplitude_per_mode(table):
    lnk, lnp = table
    cfg = model.Config(n=16, box=64.0)
    s = inputs.white_noise(16, 11).astype(np.float64)
    dl = model.linear_field(s, cfg, lnk, lnp)
    sk, dk = M.rfft3(s), M.rfft3(dl)
    kmag = np.sqrt(M.k_squared(16, 64.0))
    p = C.power_from_table(kmag, lnk, lnp)
    ratio = np.abs(dk) ** 2 / np.abs(sk) ** 2
    mask = kmag > 0
    np.testing.assert_allclose(ratio[mask], p[mask] / cfg.cell ** 3, rtol=1e-12)
    assert abs(dk[0, 0, 0]) < 1e-12


def test_linear_field_power_spectrum_matches_input(table):
    # measured P(k) of delta_L scatters around the table by sqrt(2/N_modes)
    lnk, lnp = table
    n, box = 64, 256.0
    cfg = model.Config(n=n, box=box)
    s = inputs.white_noise(n, 12).astype(np.float64)
    dl = model.linear_field(s, cfg, lnk, lnp)
    nb, kmin, kmax = 11, 2 * np.pi / box, np.pi * n / box
    pk, _, _, nm = analysis.power_spectra(dl, None, box, nb, kmin, kmax)
    # expectation of the estimator: the table averaged over each bin's modes
    m = np.fft.fftfreq(n, 1.0 / n)
    kk = 2 * np.pi / box * np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2).ravel()
    idx = np.floor((kk - kmin) / ((kmax - kmin) / nb)).astype(np.int64)
    ok = (idx >= 0) & (idx < nb)
    ptab = np.bincount(idx[ok], C.power_from_table(kk[ok], lnk, lnp), nb) / np.bincount(idx[ok], minlength=nb)
    # each independent mode appears twice among the n^3 (its conjugate), so the
    # relative scatter of a bin is sqrt(2 / N_modes)
    z = (pk / ptab - 1) / np.sqrt(2.0 / nm)
    assert np.all(np.abs(z) < 5.0)
    assert abs(np.mean(pk[2:] / ptab[2:]) - 1) < 0.05


def _s_from_linear_field(delta_l, cfg, lnk, lnp):
    amp = model.ic_amplitude(cfg, lnk, lnp)
    dk = M.rfft3(delta_l)
    sk = np.zeros_like(dk)
    np.divide(dk, amp, out=sk, where=amp > 0)
    return M.irfft3(sk, cfg.n)


def test_2lpt_plane_waves_closed_form(table):
    lnk, lnp = table
    n, box = 16, 80.0
    cfg = model.Config(n=n, box=box, lpt_order=2)
    x = np.arange(n) * box / n
    k1, k2 = 2 * np.pi / box * 2, 2 * np.pi / box * 3
    A, B = 0.3, -0.2
    X = x[:, None, None] * np.ones((1, n, n))
    Y = x[None, :, None] * np.ones((n, 1, n))
    # single wave: no second-order source, Psi1 = -A sin(k1 x)/k1 x_hat
    s = _s_from_linear_field(A * np.cos(k1 * X), cfg, lnk, lnp)
    _, _, info = model.lpt(s, cfg, lnk, lnp)
    np.testing.assert_allclose(info["psi2"], 0.0, atol=1e-15)
    np.testing.assert_allclose(info["psi1"][:, 0], (-A * np.sin(k1 * X) / k1).reshape(-1), atol=1e-13)
    np.testing.assert_allclose(info["psi1"][:, 1:], 0.0, atol=1e-13)
    # crossed waves: S = A B cos(k1 x) cos(k2 y), Psi2 = grad phi2, lap phi2 = S
    s = _s_from_linear_field(A * np.cos(k1 * X) + B * np.cos(k2 * Y), cfg, lnk, lnp)
    _, _, info = model.lpt(s, cfg, lnk, lnp)
    kk = k1 * k1 + k2 * k2
    psi2x = A * B * k1 * np.sin(k1 * X) * np.cos(k2 * Y) / kk
    psi2y = A * B * k2 * np.cos(k1 * X) * np.sin(k2 * Y) / kk
    np.testing.assert_allclose(info["psi2"][:, 0], psi2x.reshape(-1), atol=1e-14)
    np.testing.assert_allclose(info["psi2"][:, 1], psi2y.reshape(-1), atol=1e-14)
    np.testing.assert_allclose(info["psi2"][:, 2], 0.0, atol=1e-14)
    # divergence of Psi1 is -delta_L
    div = sum(M.apply_multiplier(info["psi1"][:, i].reshape(n, n, n), M.deriv(n, box, i))
              for i in range(3))
    np.testing.assert_allclose(div, -(A * np.cos(k1 * X) + B * np.cos(k2 * Y)), atol=1e-13)


def test_single_mode_force_amplitude(table):
    lnk, lnp = table
    n, box, om = 16, 64.0, 0.3
    cfg = model.Config(n=n, box=box, omega_m=om)
    ops = model._Ops(cfg, lnk, lnp)
    x = np.arange(n) * box / n
    k0 = 2 * np.pi / box * 2
    eps = 0.01
    delta = eps * np.cos(k0 * x)[None, None, :] * np.ones((n, n, 1))
    fz = M.irfft3(ops.force[2] * M.rfft3(delta), n)
    np.testing.assert_allclose(fz, -1.5 * om * eps / k0 * np.sin(k0 * x)[None, None, :] * np.ones((n, n, 1)),
                               atol=1e-15)


def test_unperturbed_lattice_and_momentum_conservation(table):
    lnk, lnp = table
    n, box = 16, 64.0
    cfg = model.Config(n=n, box=box)
    ops = model._Ops(cfg, lnk, lnp)
    f, _, delta = model.force(np.zeros((n ** 3, 3)), cfg, ops)
    assert np.all(delta == 0.0) and np.all(f == 0.0)
    s = inputs.white_noise(n, 13).astype(np.float64)
    disp, mom, _ = model.lpt(s, cfg, lnk, lnp)
    f, _, _ = model.force(disp, cfg, ops)
    # sum_p F_p = <rho, G rho> = 0 by antisymmetry of the spectral gradient
    assert np.all(np.abs(f.sum(axis=0)) < 1e-10 * np.abs(f).sum(axis=0))
    # the leapfrog therefore conserves total momentum
    d1, m1, _ = model.evolve(s, cfg, lnk, lnp)
    assert np.all(np.abs(m1.sum(axis=0) - mom.sum(axis=0)) < 1e-10 * np.abs(m1).sum(axis=0))


def test_linear_regime_growth_and_step_independence(table):
    # tiny amplitude: delta_final -> D1(1) delta_L on the largest scales,
    # the FastPM factors make the result nearly independent of n
    lnk, lnp = table
    n, box = 32, 256.0
    s = 1e-4 * inputs.white_noise(n, 14).astype(np.float64)
    out = {}
    for steps in (5, 10):
        cfg = model.Config(n=n, box=box, n_steps=steps, lpt_order=1)
        disp, mom, _ = model.evolve(s, cfg, lnk, lnp)
        out[steps] = M.rfft3(model.final_density(disp, cfg))
    cfg = model.Config(n=n, box=box)
    dl = M.rfft3(model.linear_field(s, cfg, lnk, lnp))
    idx = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (n - 1, 0, 0), (1, 1, 0)]
    for i in idx:
        r5 = out[5][i] / dl[i]
        r10 = out[10][i] / dl[i]
        # CIC assignment of a nearly unperturbed lattice and the PM force
        # window bias the largest modes by a few percent (k Delta ~ 0.2-0.3)
        assert abs(r5 - 1.0) < 0.06
        # linear exactness of the kick / drift factors: halving the step
        # changes the result by far less than a first-order scheme would
        assert abs(r10 - r5) < 1e-3


def _cases():
    return [
        model.Config(n=8, box=32.0, n_steps=3, lpt_order=2, rsd_axis=2,
                     likelihood="gaussian", bias_b=1.5, sigma=1.0, prior_weight=1.0),
        model.Config(n=8, box=40.0, n_steps=2, lpt_order=2, rsd_axis=-1,
                     likelihood="poisson", nbar_cell=2.0, prior_weight=0.5),
        # radial shift from an observer outside the box (the paper's line of sight)
        model.Config(n=8, box=32.0, n_steps=2, lpt_order=2, rsd_axis=3, observer=(16.0, 20.0, -24.0),
                     likelihood="gaussian", bias_b=1.5, sigma=1.0, prior_weight=1.0),
        # Poisson likelihood with the linear bias (rate floored at rho_floor)
        model.Config(n=8, box=40.0, n_steps=2, lpt_order=2, rsd_axis=1, likelihood="poisson", bias="linear",
                     bias_b=1.5, nbar_cell=2.0, prior_weight=0.5),
    ]


@pytest.mark.parametrize("case", [0, 1, 2, 3])
def test_gradient_brute_force_all_coordinates(table, case):
    """Central finite differences on every one of the 8^3 white-noise
    coordinates against the hand-derived adjoint."""
    lnk, lnp = table
    cfg = _cases()[case]
    n = cfg.n
    s = inputs.white_noise(n, 21).astype(np.float64)
    if cfg.likelihood == "gaussian":
        data = inputs.normal_field(n, 22).astype(np.float64)
        resp = np.ones((n, n, n))
    else:
        resp = inputs.uniform_field(n, 23, -0.5, 1.0).astype(np.float64).clip(0, None)
        data = inputs.poisson_counts(2.0 * np.ones((n, n, n)), 24).astype(np.float64)
    f0, g, _ = model.gradient(s, cfg, lnk, lnp, data, resp)
    assert f0 == pytest.approx(model.loss(s, cfg, lnk, lnp, data, resp)[0], rel=1e-14)
    eps = 1e-6
    fd = np.empty(n ** 3)
    for i in range(n ** 3):
        sp, sm = s.copy(), s.copy()
        sp.flat[i] += eps
        sm.flat[i] -= eps
        fd[i] = (model.loss(sp, cfg, lnk, lnp, data, resp)[0]
                 - model.loss(sm, cfg, lnk, lnp, data, resp)[0]) / (2 * eps)
    err = np.abs(fd - g.reshape(-1))
    scale = np.abs(g).max()
    bad = err > 1e-6 * scale + 1e-6 * np.abs(g.reshape(-1))
    # a coordinate whose difference straddles a CIC cell face may disagree;
    # no more than a handful of those
    assert np.count_nonzero(bad) <= 3
    assert np.linalg.norm(fd - g.reshape(-1)) / np.linalg.norm(g) < 1e-6


def test_gradient_of_density_cotangent_and_loss_weight(table):
    lnk, lnp = table
    cfg = model.Config(n=8, box=32.0, n_steps=2, rsd_axis=0)
    n = cfg.n
    s = inputs.white_noise(n, 31).astype(np.float64)
    data = inputs.normal_field(n, 32).astype(np.float64)
    resp = np.ones((n, n, n))
    cot = inputs.normal_field(n, 33).astype(np.float64)
    _, g, _ = model.gradient(s, cfg, lnk, lnp, data, resp, loss_weight=0.0, cot_delta=cot)

    def fun(x):
        disp, mom, _ = model.evolve(x, cfg, lnk, lnp)
        return np.sum(cot * model.final_density(model.observed_positions(disp, mom, cfg), cfg))
    rng = np.random.default_rng(34)
    for _ in range(3):
        v = rng.standard_normal((n, n, n))
        e = 1e-6
        fd = (fun(s + e * v) - fun(s - e * v)) / (2 * e)
        assert fd == pytest.approx(np.sum(g * v), rel=1e-7)
    _, g2, _ = model.gradient(s, cfg, lnk, lnp, data, resp, loss_weight=2.0)
    _, g1, _ = model.gradient(s, cfg, lnk, lnp, data, resp, loss_weight=1.0)
    np.testing.assert_allclose(g2, 2 * g1, rtol=1e-12, atol=1e-12)


def test_loss_at_zero_field_closed_form(table):
    lnk, lnp = table
    n = 8
    s = np.zeros((n, n, n))
    data = inputs.normal_field(n, 41).astype(np.float64)
    resp = inputs.uniform_field(n, 42, 0.0, 1.0).astype(np.float64)
    cfg = model.Config(n=n, box=32.0, n_steps=2, likelihood="gaussian", sigma=0.7)
    f, _ = model.loss(s, cfg, lnk, lnp, data, resp)
    assert f == pytest.approx(0.5 * np.sum(resp * data ** 2) / 0.7 ** 2, rel=1e-13)
    cfgp = model.Config(n=n, box=32.0, n_steps=2, likelihood="poisson", nbar_cell=3.0)
    counts = inputs.poisson_counts(np.ones((n, n, n)), 43).astype(np.float64)
    f, _ = model.loss(s, cfgp, lnk, lnp, counts, resp)
    g0 = 1.0 / (1.0 + np.exp(-3.0 * (0.0 - 1.2)))      # (1+0)^0.7 sigmoid(K(0 - 1.2))
    lam = resp * 3.0 * g0
    m = resp > 0
    assert f == pytest.approx(np.sum(lam[m] - counts[m] * np.log(lam[m])), rel=1e-12)


def test_force_vjp_dot_product(table):
    lnk, lnp = table
    cfg = model.Config(n=8, box=32.0)
    ops = model._Ops(cfg, lnk, lnp)
    n = cfg.n
    rng = np.random.default_rng(51)
    disp = rng.normal(0, 3.0, (n ** 3, 3))
    v = rng.standard_normal((n ** 3, 3))
    w = rng.standard_normal((n ** 3, 3))
    e = 1e-6
    jv = (model.force(disp + e * v, cfg, ops)[0] - model.force(disp - e * v, cfg, ops)[0]) / (2 * e)
    assert np.sum(jv * w) == pytest.approx(np.sum(v * model.force_vjp(disp, w, cfg, ops)), rel=1e-6)


def test_rsd_kaiser_limit(table):
    # linear theory (Kaiser 1987): a plane-parallel shift multiplies a mode
    # along the line of sight by 1 + f, f = dlnD1/dlna, and leaves modes
    # perpendicular to it unchanged
    lnk, lnp = table
    n, box = 32, 256.0
    s = 1e-4 * inputs.white_noise(n, 15).astype(np.float64)
    cfg = model.Config(n=n, box=box, n_steps=5, lpt_order=1, rsd_axis=2)
    disp, mom, _ = model.evolve(s, cfg, lnk, lnp)
    real = M.rfft3(model.final_density(disp, cfg))
    red = M.rfft3(model.final_density(model.observed_positions(disp, mom, cfg), cfg))
    f = C.growth([1.0], cfg.omega_m)["dD1"][0]         # a dD1/da / D1 at a = 1
    # the fundamental line-of-sight mode (higher modes feel the grid)
    assert abs(red[0, 0, 1] / real[0, 0, 1] - (1.0 + f)) < 0.01 * (1.0 + f)
    # modes with k_z = 0 see the z-integrated density, which a shift along z
    # cannot change (the CIC weights of a particle sum to one along z)
    for i in [(1, 0, 0), (0, 2, 0), (3, 5, 0)]:
        assert abs(red[i] / real[i] - 1.0) < 1e-9
    # no momentum, no shift
    np.testing.assert_array_equal(model.observed_positions(disp, 0 * mom, cfg), disp)


def test_radial_rsd_closed_forms():
    """Radial shift: zero momentum leaves positions unchanged; for a distant
    observer on the -z side it tends to the plane-parallel shift along z
    (error ~ transverse distance / observer distance); the shift is along the
    line of sight with length c (p . d)."""
    n, box = 8, 32.0
    rng = np.random.default_rng(5)
    disp = rng.normal(0, 0.5, (n ** 3, 3))
    mom = rng.normal(0, 1.0, (n ** 3, 3))
    far = model.Config(n=n, box=box, rsd_axis=3, observer=(16.0, 16.0, -1e7))
    pp = model.Config(n=n, box=box, rsd_axis=2)
    np.testing.assert_array_equal(model.observed_positions(disp, 0 * mom, far), disp)
    a, b = model.observed_positions(disp, mom, far), model.observed_positions(disp, mom, pp)
    assert np.abs(a - b).max() < 1e-4 * np.abs(mom).max()
    near = model.Config(n=n, box=box, rsd_axis=3, observer=(10.0, -5.0, -40.0))
    shift = model.observed_positions(disp, mom, near) - disp
    r = (np.array([[i, j, l] for i in range(n) for j in range(n) for l in range(n)], float) * (box / n)
         + disp - np.array(near.observer))
    d = r / np.linalg.norm(r, axis=1)[:, None]
    c = model.rsd_coefficient(near)
    np.testing.assert_allclose(shift, c * np.sum(mom * d, axis=1)[:, None] * d, rtol=1e-12, atol=1e-12)


def test_radial_rsd_vjp_dot_product(table):
    """<J v, w> = <v, J^T w> for the radial shift's Jacobian wrt (disp, mom),
    by central differences along random directions."""
    n, box = 8, 32.0
    cfg = model.Config(n=n, box=box, rsd_axis=3, observer=(12.0, 40.0, -30.0))
    rng = np.random.default_rng(6)
    disp = rng.normal(0, 0.5, (n ** 3, 3))
    mom = rng.normal(0, 1.0, (n ** 3, 3))
    w = rng.standard_normal((n ** 3, 3))
    xb, pb = model.observed_positions_vjp(disp, mom, w, cfg)
    for _ in range(3):
        vx, vp = rng.standard_normal((n ** 3, 3)), rng.standard_normal((n ** 3, 3))
        h = 1e-6
        jv = (model.observed_positions(disp + h * vx, mom + h * vp, cfg)
              - model.observed_positions(disp - h * vx, mom - h * vp, cfg)) / (2 * h)
        lhs = np.sum(jv * w)
        rhs = np.sum(vx * xb) + np.sum(vp * pb)
        assert abs(lhs - rhs) < 1e-7 * abs(rhs)


def test_comoving_distance_and_inverse():
    """chi(a) for Omega_m = 1 is 2 (c/H0)(1 - sqrt(a)) (closed form); the
    table inverse returns a to the linear-interpolation error of its grid."""
    from oracle import cosmology as OC
    a = np.array([0.5, 0.63, 0.8, 0.9, 0.97, 1.0])
    np.testing.assert_allclose(OC.comoving_distance(a, 1.0), 2 * OC.C_OVER_H0 * (1 - np.sqrt(a)), rtol=1e-10,
                               atol=1e-9)
    at, ct = OC.distance_table(0.25)
    aa = np.linspace(0.52, 0.999, 37)
    back, slope = OC.dist_to_scale_factor(OC.comoving_distance(aa, 0.25), at, ct)
    assert np.abs(back - aa).max() < 1e-7
    # slope = 1 / (dchi/da) = -a^2 E / (c/H0)
    np.testing.assert_allclose(slope, -aa ** 2 * OC.efunc(aa, 0.25) / OC.C_OVER_H0, rtol=2e-3)


def test_lightcone_static_snapshots_closed_form():
    """With identical snapshots the observed displacement is the snapshot plus
    the radial shift at a_i = DistToScaleFactor(|q + x - o|)."""
    from oracle import cosmology as OC
    n, box = 8, 64.0
    cfg = model.Config(n=n, box=box, lightcone=True, observer=(30.0, 40.0, -450.0))
    rng = np.random.default_rng(8)
    x = rng.normal(0, 1.0, (n ** 3, 3))
    p = rng.normal(0, 2.0, (n ** 3, 3))
    X, P = np.stack([x, x, x]), np.stack([p, p, p])
    tab = OC.distance_table(cfg.omega_m)
    obs = model.lightcone_observed(X, P, cfg, tab)
    q = np.array([[i, j, l] for i in range(n) for j in range(n) for l in range(n)], float) * (box / n)
    r = q + x - np.array(cfg.observer)
    d = np.linalg.norm(r, axis=1)
    a, _ = OC.dist_to_scale_factor(d, *tab)
    assert (a > 0.8).all() and (a < 0.9).all()
    u = r / d[:, None]
    s = 1.0 / (a * a * OC.efunc(a, cfg.omega_m))
    np.testing.assert_allclose(obs, x + (s * np.sum(p * u, axis=1))[:, None] * u, rtol=1e-12, atol=1e-12)


def test_lightcone_vjp_dot_product():
    """<J v, w> = <v, J^T w> for the lightcone map wrt all snapshot positions
    and momenta (iterations, interpolation and shift), central differences."""
    from oracle import cosmology as OC
    n, box = 8, 64.0
    cfg = model.Config(n=n, box=box, lightcone=True, observer=(30.0, 40.0, -450.0))
    rng = np.random.default_rng(9)
    base = rng.normal(0, 1.0, (n ** 3, 3))
    X = np.stack([base + rng.normal(0, 3.0, base.shape) * t for t in (0.0, 0.5, 1.0)])
    P = rng.normal(0, 2.0, (3, n ** 3, 3))
    tab = OC.distance_table(cfg.omega_m)
    w = rng.standard_normal((n ** 3, 3))
    Xb, Pb = model.lightcone_vjp(X, P, w, cfg, tab)
    for _ in range(3):
        vx, vp = rng.standard_normal(X.shape), rng.standard_normal(P.shape)
        h = 1e-6
        jv = (model.lightcone_observed(X + h * vx, P + h * vp, cfg, tab)
              - model.lightcone_observed(X - h * vx, P - h * vp, cfg, tab)) / (2 * h)
        lhs, rhs = np.sum(jv * w), np.sum(vx * Xb) + np.sum(vp * Pb)
        assert abs(lhs - rhs) < 1e-6 * abs(rhs), (lhs, rhs)


def test_lightcone_gradient_brute_force(table):
    """Central differences on all 512 coordinates of an 8^3 lightcone case
    (snapshots at a = 0.8, 0.9, 1 of a 9-step run, observer 450 Mpc/h away)."""
    lnk, lnp = table
    cfg = model.Config(n=8, box=64.0, n_steps=9, lpt_order=2, lightcone=True, observer=(30.0, 40.0, -450.0),
                       likelihood="gaussian", bias_b=1.5, sigma=1.0, prior_weight=1.0)
    n = cfg.n
    s = inputs.white_noise(n, 41).astype(np.float64)
    data = inputs.normal_field(n, 42).astype(np.float64)
    resp = np.ones((n, n, n))
    f0, g, _ = model.gradient(s, cfg, lnk, lnp, data, resp)
    assert f0 == pytest.approx(model.loss(s, cfg, lnk, lnp, data, resp)[0], rel=1e-14)
    eps = 1e-6
    fd = np.empty(n ** 3)
    for i in range(n ** 3):
        sp, sm = s.copy(), s.copy()
        sp.flat[i] += eps
        sm.flat[i] -= eps
        fd[i] = (model.loss(sp, cfg, lnk, lnp, data, resp)[0] - model.loss(sm, cfg, lnk, lnp, data, resp)[0]) / (2 * eps)
    bad = np.abs(fd - g.reshape(-1)) > 1e-6 * np.abs(g).max() + 1e-6 * np.abs(g.reshape(-1))
    assert np.count_nonzero(bad) <= 3
    assert np.linalg.norm(fd - g.reshape(-1)) / np.linalg.norm(g) < 1e-6
