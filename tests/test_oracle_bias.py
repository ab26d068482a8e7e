"""Pins of the oracle's bias models and likelihoods (Sec. 2.2.1 item 4,
Sec. 2.2.2, Eq. galaxy_bias) in all four pairings: each -log L equals the
negative log of scipy's Poisson pmf / normal pdf summed over the observed
cells, less the data-only constants (log N!, the Gaussian normaliser), and
each derivative equals central differences of that library value, cell by
cell.  The "auto" bias resolves to the pairs Sec. 2.2.2 describes."""
import dataclasses

import numpy as np
import pytest
from scipy import special, stats

from oracle import model


def _fields(n=4096, seed=5):
    rng = np.random.default_rng(seed)
    delta = rng.uniform(-0.95, 4.0, n)
    delta[:64] = rng.uniform(-0.999, -0.9, 64)     # deep voids: 1 + b delta below the floor for b > 1
    resp = rng.uniform(-0.3, 1.0, n).clip(0, None)  # ~23% unobserved cells (R = 0)
    return delta, resp


def _mean(delta, cfg, kind):
    """The model's mean per unit response, from Eq. galaxy_bias (or the
    linear model) and the floor."""
    if kind == "linear":
        return cfg.nbar_cell * np.maximum(1.0 + cfg.bias_b * delta, cfg.rho_floor)
    return (cfg.nbar_cell * np.maximum(1.0 + delta, cfg.rho_floor) ** cfg.alpha
            * special.expit(cfg.K * (delta - cfg.delta_th)))


def _library_terms(delta, data, resp, cfg, kind):
    """Per-cell -log L from scipy's densities, constants removed."""
    m = resp > 0
    out = np.zeros_like(delta)
    if cfg.likelihood == "poisson":
        lam = resp[m] * _mean(delta[m], cfg, kind)
        out[m] = -stats.poisson.logpmf(data[m], lam) - special.gammaln(data[m] + 1.0)
    else:
        f = cfg.bias_b * delta[m] if kind == "linear" else _mean(delta[m], cfg, kind)
        sd = cfg.sigma / np.sqrt(resp[m])
        out[m] = -stats.norm.logpdf(data[m], f, sd) - 0.5 * np.log(2.0 * np.pi * sd ** 2)
    return out


CFG = model.Config(n=16, box=64.0, bias_b=1.5, sigma=0.7, alpha=0.7, delta_th=1.2, K=3.0, nbar_cell=2.5,
                   rho_floor=1e-3)


@pytest.mark.parametrize("lik,bias", [("gaussian", "linear"), ("gaussian", "powerlaw_sigmoid"),
                                      ("poisson", "linear"), ("poisson", "powerlaw_sigmoid")])
def test_likelihood_matches_library_densities(lik, bias):
    cfg = dataclasses.replace(CFG, likelihood=lik, bias=bias)
    delta, resp = _fields()
    rng = np.random.default_rng(6)
    if lik == "poisson":
        data = rng.poisson(resp * 1.7).astype(np.float64)
    else:
        data = rng.normal(0.5, 1.5, delta.size)
    val, grad = model.likelihood_terms(delta, data, resp, cfg)
    ref = _library_terms(delta, data, resp, cfg, bias)
    assert val == pytest.approx(ref.sum(), rel=1e-12)
    eps = 1e-6
    fd = (_library_terms(delta + eps, data, resp, cfg, bias)
          - _library_terms(delta - eps, data, resp, cfg, bias)) / (2 * eps)
    # away from the floor's kink the derivative is smooth
    kink = np.abs(1.0 + (cfg.bias_b if bias == "linear" else 1.0) * delta - cfg.rho_floor) < 1e-4
    ok = ~kink
    np.testing.assert_allclose(grad[ok], fd[ok], rtol=1e-6, atol=1e-7 * np.abs(fd).max())
    assert np.all(grad[resp == 0] == 0)
    if lik == "poisson" and bias == "linear":
        below = 1.0 + cfg.bias_b * delta < cfg.rho_floor
        assert below.sum() > 10 and np.all(grad[below] == 0)


@pytest.mark.parametrize("lik,bias", [("gaussian", "linear"), ("gaussian", "powerlaw_sigmoid"),
                                      ("poisson", "linear"), ("poisson", "powerlaw_sigmoid")])
def test_model_mean(lik, bias):
    """The mock rate: R times the mean of Eq. galaxy_bias (or the linear
    model) for the Poisson, the biased field for the Gaussian; the Gaussian
    likelihood vanishes at data equal to it."""
    cfg = dataclasses.replace(CFG, likelihood=lik, bias=bias)
    delta, resp = _fields(1024, 11)
    mu = model.model_mean(delta, resp, cfg)
    if lik == "poisson":
        np.testing.assert_allclose(mu, np.where(resp > 0, resp * _mean(delta, cfg, bias), 0.0), rtol=1e-14)
    else:
        ref = cfg.bias_b * delta if bias == "linear" else _mean(delta, cfg, bias)
        np.testing.assert_allclose(mu, ref, rtol=1e-14)
        val, grad = model.likelihood_terms(delta, mu, resp, cfg)
        assert val == 0.0 and np.all(grad == 0.0)


def test_auto_bias_is_the_papers_pairing():
    delta, resp = _fields(512, 7)
    data = np.random.default_rng(8).poisson(resp).astype(np.float64)
    for lik, kind in (("gaussian", "linear"), ("poisson", "powerlaw_sigmoid")):
        a = model.likelihood_terms(delta, data, resp, dataclasses.replace(CFG, likelihood=lik))
        b = model.likelihood_terms(delta, data, resp, dataclasses.replace(CFG, likelihood=lik, bias=kind))
        assert a[0] == b[0] and np.array_equal(a[1], b[1])
    with pytest.raises(ValueError):
        model.bias_kind(dataclasses.replace(CFG, bias="quadratic"))


def test_linear_poisson_is_the_power_law_at_alpha_one_and_flat_sigmoid():
    """b = 1: max(1 + delta, floor) equals the power law with alpha = 1 times
    a sigmoid at K = 0 (= 1/2) with twice the normalisation."""
    delta, resp = _fields(2048, 9)
    data = np.random.default_rng(10).poisson(resp * 2).astype(np.float64)
    lin = dataclasses.replace(CFG, likelihood="poisson", bias="linear", bias_b=1.0, nbar_cell=1.3)
    pw = dataclasses.replace(CFG, likelihood="poisson", bias="powerlaw_sigmoid", alpha=1.0, K=0.0, nbar_cell=2.6)
    a = model.likelihood_terms(delta, data, resp, lin)
    b = model.likelihood_terms(delta, data, resp, pw)
    assert a[0] == pytest.approx(b[0], rel=1e-13)
    np.testing.assert_allclose(a[1], b[1], rtol=1e-12, atol=1e-14)
