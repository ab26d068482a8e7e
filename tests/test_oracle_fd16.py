"""Brute-force pin of the oracle's hand-derived gradient at 16^3: central
finite differences of the loss on every one of the 4096 white-noise
coordinates (eps = 1e-6, FP64), 2LPT and three leapfrog steps, against
``model.gradient``.  The differences run in a pool of worker processes
started with ``spawn``; each worker runs the single-threaded oracle on its
share of the coordinates.

A coordinate whose +-eps perturbation moves some particle across a CIC cell
face sees a kink of the piecewise-linear CIC weights (the floor convention of
the derivative at a face), so its central difference may disagree with the
one-sided derivative; such coordinates are rare and the test allows a few.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import cosmology as C
from oracle import model
from paper_2604_26823_gb300 import inputs

pytestmark = pytest.mark.slow

N = 16
EPS = 1e-6

CASES = {
    # Gaussian likelihood, linear bias, plane-parallel RSD along z, prior on
    "gaussian_rsd": dict(n=N, box=64.0, n_steps=3, lpt_order=2, rsd_axis=2, likelihood="gaussian",
                         bias_b=1.5, sigma=1.0, prior_weight=1.0),
    # masked Poisson likelihood with the power-law + sigmoid bias
    "poisson_mask": dict(n=N, box=64.0, n_steps=3, lpt_order=2, rsd_axis=-1, likelihood="poisson",
                         nbar_cell=2.0, prior_weight=0.5),
}


def _inputs(name):
    kw = CASES[name]
    s = inputs.white_noise(N, 21).astype(np.float64)
    if kw["likelihood"] == "gaussian":
        data = inputs.normal_field(N, 22).astype(np.float64)
        resp = np.ones((N, N, N))
    else:
        resp = inputs.uniform_field(N, 23, -0.5, 1.0).astype(np.float64).clip(0, None)
        data = inputs.poisson_counts(2.0 * np.ones((N, N, N)), 24).astype(np.float64)
    return s, data, resp


def _fd_chunk(args):
    """Central differences of the oracle loss on the given coordinates."""
    name, idx = args
    lnk, lnp = C.linear_power_table()
    cfg = model.Config(**CASES[name])
    s, data, resp = _inputs(name)
    out = np.empty(len(idx))
    for j, i in enumerate(idx):
        sp, sm = s.copy(), s.copy()
        sp.flat[i] += EPS
        sm.flat[i] -= EPS
        out[j] = (model.loss(sp, cfg, lnk, lnp, data, resp)[0]
                  - model.loss(sm, cfg, lnk, lnp, data, resp)[0]) / (2 * EPS)
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_gradient_brute_force_all_4096_coordinates(name):
    lnk, lnp = C.linear_power_table()
    cfg = model.Config(**CASES[name])
    s, data, resp = _inputs(name)
    f0, g, _ = model.gradient(s, cfg, lnk, lnp, data, resp)
    assert f0 == pytest.approx(model.loss(s, cfg, lnk, lnp, data, resp)[0], rel=1e-14)
    workers = max(1, min(8, os.cpu_count() or 1))
    chunks = np.array_split(np.arange(N ** 3), 4 * workers)
    with mp.get_context("spawn").Pool(workers) as pool:
        fd = np.concatenate(pool.map(_fd_chunk, [(name, c) for c in chunks]))
    g = g.reshape(-1)
    err = np.abs(fd - g)
    bad = err > 1e-6 * np.abs(g).max() + 1e-6 * np.abs(g)
    print(f"{name}: relative L2 of FD vs adjoint {np.linalg.norm(fd - g) / np.linalg.norm(g):.2e}, "
          f"max |err| / max |g| {err.max() / np.abs(g).max():.2e}, coordinates off {np.count_nonzero(bad)}")
    assert np.count_nonzero(bad) <= 4
    assert np.linalg.norm(fd - g) / np.linalg.norm(g) < 1e-6
