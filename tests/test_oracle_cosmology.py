"""Pins of the oracle's background cosmology, growth and leapfrog factors
against closed forms (Einstein-de Sitter, Heath 1977) and independent
quadratures."""
import numpy as np
import pytest
from scipy import integrate

from oracle import cosmology as C


def test_eds_growth_closed_form():
    # Omega_m = 1: D1 = a, D2 = -3/7 a^2, Gp1 = a^3 E dD1/da = a^{3/2}
    a = np.array([0.05, 0.1, 0.37, 0.8, 1.0])
    g = C.growth(a, 1.0)
    np.testing.assert_allclose(g["D1"], a, rtol=1e-11)
    np.testing.assert_allclose(g["D2"], -3.0 / 7.0 * a ** 2, rtol=1e-10)
    np.testing.assert_allclose(g["dD1"], np.ones_like(a), rtol=1e-10)
    np.testing.assert_allclose(g["Gp1"], a ** 1.5, rtol=1e-10)
    np.testing.assert_allclose(g["Gp2"], a ** 3 * a ** -1.5 * (-6.0 / 7.0) * a, rtol=1e-10)


@pytest.mark.parametrize("om", [0.25, 0.315])
def test_lcdm_growth_matches_heath_integral(om):
    a = np.array([0.1, 0.28, 0.55, 0.9, 1.0])
    g = C.growth(a, om)
    np.testing.assert_allclose(g["D1"], C.heath_growth(a, om), rtol=1e-10)


def test_lcdm_second_order_growth_vs_bouchet_fit():
    # D2 ~ -3/7 Om(a)^(-1/143) D1^2 (Bouchet et al. 1995), better than 1%
    a = np.array([0.3, 0.6, 1.0])
    om = 0.25
    g = C.growth(a, om)
    fit = -3.0 / 7.0 * C.omega_m_of_a(a, om) ** (-1.0 / 143.0) * g["D1"] ** 2
    np.testing.assert_allclose(g["D2"], fit, rtol=3e-3)
    # and a sign or factor error would break the EdS limit at early times
    early = C.growth([0.01], om)
    assert abs(early["D2"][0] / (-3.0 / 7.0 * early["D1"][0] ** 2) - 1) < 1e-3


def test_momentum_growth_is_integral_of_force_growth():
    # dGp/da = Gf / (a^2 E) with Gf = 1.5 Om D1: checks Gp and the ODE
    # against an independent quadrature of the Heath growth factor.
    om = 0.25
    a0, a1 = 0.1, 0.73
    g = C.growth([a0, a1], om)
    val, _ = integrate.quad(lambda t: 1.5 * om * C.heath_growth(t, om)[0] /
                            (t * t * C.efunc(t, om)), a0, a1, epsrel=1e-12)
    assert abs((g["Gp1"][1] - g["Gp1"][0]) / val - 1) < 1e-9


def test_leapfrog_factors_exact_for_linear_growth():
    # x = D1 Psi, p = Gp Psi, F = Gf Psi is reproduced exactly by the
    # schedule; with an independent quadrature for the integrals.
    om, ai, n = 0.25, 0.1, 5
    sch = C.leapfrog_schedule(ai, n, om)
    a = sch["a"]
    assert a[0] == ai and a[-1] == 1.0 and np.allclose(np.diff(a), (1 - ai) / n)
    d1 = lambda t: C.heath_growth(t, om)[0]
    gp = lambda t: C.growth([t], om)["Gp1"][0]
    for k in range(n):
        ah = 0.5 * (a[k] + a[k + 1])
        # kick: Ka Gf(a_k) = int_{a_k}^{a_h} Gf/(a^2 E)
        kick, _ = integrate.quad(lambda t: 1.5 * om * d1(t) / (t * t * C.efunc(t, om)),
                                 a[k], ah, epsrel=1e-12)
        assert abs(sch["Ka"][k] * 1.5 * om * d1(a[k]) / kick - 1) < 1e-8
        kick2, _ = integrate.quad(lambda t: 1.5 * om * d1(t) / (t * t * C.efunc(t, om)),
                                  ah, a[k + 1], epsrel=1e-12)
        assert abs(sch["Kb"][k] * 1.5 * om * d1(a[k + 1]) / kick2 - 1) < 1e-8
        # drift: Dr Gp(a_h) = D1(a_{k+1}) - D1(a_k)
        assert abs(sch["Dr"][k] * gp(ah) / (d1(a[k + 1]) - d1(a[k])) - 1) < 1e-9


def test_power_table_normalisation_and_limits():
    lnk, lnp = C.linear_power_table(omega_m=0.25, omega_b=0.045, h=0.73, sigma8=0.9, n_s=1.0)
    assert lnk.size == 512
    assert abs(np.exp(lnk[0]) - 1e-4) < 1e-12 and abs(np.exp(lnk[-1]) - 1e2) < 1e-9
    # sigma8 recomputed from the table by an independent trapezoid in ln k
    k = np.exp(np.linspace(np.log(1e-4), np.log(1e2), 200001))
    pk = C.power_from_table(k, lnk, lnp)
    x = k * 8.0
    w = 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3
    s2 = np.trapezoid(k ** 3 * pk * w * w, np.log(k)) / (2 * np.pi ** 2)
    assert abs(np.sqrt(s2) - 0.9) < 2e-4
    # transfer function -> 1 as k -> 0; primordial slope n_s at low k
    assert abs(C.eh98_nowiggle_transfer(1e-7, 0.25, 0.045, 0.73) - 1.0) < 1e-6
    slope = (lnp[1] - lnp[0]) / (lnk[1] - lnk[0])
    assert abs(slope - 1.0) < 0.01
    # turnover: P(k) peaks at k ~ 0.01-0.03 h/Mpc for Omega_m h ~ 0.18
    kpk = np.exp(lnk[np.argmax(lnp)])
    assert 0.008 < kpk < 0.04
    # interpolation clamps at the table ends and is exact on the nodes
    assert C.power_from_table(np.exp(lnk[10]), lnk, lnp) == pytest.approx(np.exp(lnp[10]), rel=1e-13)
    assert C.power_from_table(1e3, lnk, lnp) == pytest.approx(np.exp(lnp[-1]), rel=1e-13)
