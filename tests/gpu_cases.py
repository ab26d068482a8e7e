"""Shared set-up of the GPU parity tests: configurations mirrored on both
sides, seeded inputs, and cached oracle results (the oracle runs once per
configuration per test session)."""
import functools

import numpy as np

from oracle import cosmology as OC
from oracle import model as OM
from paper_2604_26823_gb300 import inputs


@functools.lru_cache(maxsize=None)
def table():
    return OC.linear_power_table()


# name -> (api Config kwargs); the oracle receives the same values
CASES = {
    # 32^3 particles in a 128 Mpc/h box, 2LPT to a = 0.1, 5 steps, b = 1.5 Gaussian, full box
    "small": dict(n=32, box=128.0, n_steps=5, lpt_order=2, rsd_axis=-1, likelihood="gaussian",
                  bias_b=1.5, sigma=1.0, prior_weight=1.0),
    # 128^3 in 512 Mpc/h, 10 steps, redshift-space shift along z
    "rsd128": dict(n=128, box=512.0, n_steps=10, lpt_order=2, rsd_axis=2, likelihood="gaussian",
                   bias_b=1.5, sigma=1.0, prior_weight=1.0),
    # masked Poisson likelihood with the power-law + sigmoid bias, 64^3 in 125 Mpc/h
    "poisson64": dict(n=64, box=125.0, n_steps=4, lpt_order=2, rsd_axis=-1, likelihood="poisson",
                      nbar_cell=0.5, alpha=0.7, delta_th=1.2, K=3.0, rho_floor=1e-3, prior_weight=1.0),
    # radial redshift-space shift seen from an observer outside the box (the
    # paper's line of sight), masked Poisson likelihood, 64^3 in 125 Mpc/h
    "radial64": dict(n=64, box=125.0, n_steps=4, lpt_order=2, rsd_axis=3, observer=(62.5, 62.5, -60.0),
                     likelihood="poisson", nbar_cell=0.5, alpha=0.7, delta_th=1.2, K=3.0, rho_floor=1e-3,
                     prior_weight=1.0),
    # observed on the past light cone (snapshots at a = 0.8, 0.9, 1 of a 9-step
    # run from a = 0.1; the box spans comoving distances 260-400 Mpc/h, across
    # the a = 0.9 snapshot), 32^3 in 128 Mpc/h, linear bias
    "lightcone32": dict(n=32, box=128.0, n_steps=9, lpt_order=2, rsd_axis=3, lightcone=True,
                        observer=(64.0, 64.0, -260.0), likelihood="gaussian", bias_b=1.5, sigma=1.0,
                        prior_weight=1.0),
    # each bias model with the other likelihood, 32^3 in 128 Mpc/h, 5 steps:
    # masked Poisson with the linear bias (rate max(1 + b delta, rho_floor)),
    # RSD along y; Gaussian on nbar times the power law + sigmoid
    "poislin32": dict(n=32, box=128.0, n_steps=5, lpt_order=2, rsd_axis=1, likelihood="poisson", bias="linear",
                      bias_b=1.5, nbar_cell=0.5, rho_floor=1e-3, prior_weight=1.0),
    "gausspl32": dict(n=32, box=128.0, n_steps=5, lpt_order=2, rsd_axis=-1, likelihood="gaussian",
                      bias="powerlaw_sigmoid", sigma=1.0, nbar_cell=2.0, alpha=0.7, delta_th=1.2, K=3.0,
                      rho_floor=1e-3, prior_weight=1.0),
    # Zel'dovich start, RSD along x, 16^3 (single-tile meshes)
    "tiny": dict(n=16, box=48.0, n_steps=3, lpt_order=1, rsd_axis=0, likelihood="gaussian",
                 bias_b=1.2, sigma=0.8, prior_weight=0.5),
}


def oracle_config(kw):
    keys = ("n", "box", "n_steps", "lpt_order", "rsd_axis", "observer", "lightcone", "likelihood", "bias", "bias_b",
            "sigma",
            "alpha",
            "delta_th", "K", "nbar_cell", "rho_floor", "prior_weight")
    return OM.Config(**{k: kw[k] for k in keys if k in kw})


@functools.lru_cache(maxsize=None)
def case_inputs(name):
    """(s, data, R) as float64 numpy arrays (exactly representable in float32)."""
    kw = CASES[name]
    n = kw["n"]
    s = inputs.white_noise(n, 2).astype(np.float64)
    if kw["likelihood"] == "gaussian":
        data = inputs.normal_field(n, 3).astype(np.float64)
        resp = np.ones((n, n, n)) if name != "tiny" else inputs.uniform_field(n, 4, 0.0, 1.0).astype(np.float64)
    else:
        sel = inputs.survey_selection(n, kw["box"], 4, observer=(62.5, 62.5, -60.0), r_scale=70.0)
        resp = sel.astype(np.float64)
        data = inputs.poisson_counts(0.5 * resp * 1.3, 5).astype(np.float64)
    return s, data, resp


@functools.lru_cache(maxsize=None)
def oracle_gradient(name):
    cfg = oracle_config(CASES[name])
    s, data, resp = case_inputs(name)
    lnk, lnp = table()
    return OM.gradient(s, cfg, lnk, lnp, data, resp)


@functools.lru_cache(maxsize=None)
def oracle_gradient_single_fft(name, lib="scipy"):
    """The oracle's gradient with every FFT step evaluated in single precision
    (scipy.fft or numpy.fft on float32 data): an independent FP32 evaluation
    of the same algorithm."""
    import scipy.fft as sf
    from oracle import mesh as OMesh
    f = sf if lib == "scipy" else np.fft
    r64, i64 = OMesh.rfft3, OMesh.irfft3
    OMesh.rfft3 = lambda x: f.rfftn(np.asarray(x, np.float32)).astype(np.complex128)
    OMesh.irfft3 = lambda fk, n: f.irfftn(np.asarray(fk, np.complex64), s=(n, n, n),
                                          axes=(0, 1, 2)).astype(np.float64)
    try:
        cfg = oracle_config(CASES[name])
        s, data, resp = case_inputs(name)
        lnk, lnp = table()
        return OM.gradient(s, cfg, lnk, lnp, data, resp)
    finally:
        OMesh.rfft3, OMesh.irfft3 = r64, i64


def _perturbed(name, amp, seed):
    s, _, _ = case_inputs(name)
    return s + np.random.default_rng(seed).standard_normal(s.shape) * np.abs(s) * amp


def perturbation_for_trajectory_error(name, traj_err):
    """Relative amplitude a of input noise a |s| N(0,1) whose FP64 trajectory
    (final displacement) deviates from the unperturbed one by traj_err in
    relative L2 (the deviation is linear in a at these sizes)."""
    cfg = oracle_config(CASES[name])
    lnk, lnp = table()
    a0 = 2.0 ** -22
    d, _, _ = OM.evolve(_perturbed(name, a0, 10), cfg, lnk, lnp)
    return a0 * traj_err / rel_l2(d, oracle_evolve(name)[0])


def oracle_gradient_perturbed(name, amp, seed):
    """The FP64 oracle's gradient at s + amp |s| N(0,1) (seeded)."""
    cfg = oracle_config(CASES[name])
    _, data, resp = case_inputs(name)
    lnk, lnp = table()
    return OM.gradient(_perturbed(name, amp, seed), cfg, lnk, lnp, data, resp)


def fp32_error_levels(name, traj_err=None, seeds=(11, 12)):
    """Relative L2 distance to the FP64 oracle's gradient of independent
    single-precision-level evaluations: the oracle with scipy's and with
    numpy's FP32 FFTs and, when traj_err (the FP32 path's own final
    displacement error) is given, the FP64 oracle from inputs perturbed so
    that its trajectory deviates by that same amount.  The CIC weight
    derivative jumps at cell faces, so on a noise-dominated adjoint each such
    evaluation's error is set by the few particles whose derivative branch
    flips -- a random quantity; these evaluations sample its spread."""
    _, rg, _ = oracle_gradient(name)
    out = {"scipy_fft32": rel_l2(oracle_gradient_single_fft(name, "scipy")[1], rg),
           "numpy_fft32": rel_l2(oracle_gradient_single_fft(name, "numpy")[1], rg)}
    if traj_err is not None:
        amp = perturbation_for_trajectory_error(name, traj_err)
        for sd in seeds:
            out[f"traj_matched_{sd}"] = rel_l2(oracle_gradient_perturbed(name, amp, sd)[1], rg)
    return out


@functools.lru_cache(maxsize=None)
def oracle_evolve(name):
    cfg = oracle_config(CASES[name])
    s, _, _ = case_inputs(name)
    lnk, lnp = table()
    disp, mom, _ = OM.evolve(s, cfg, lnk, lnp)
    return disp, mom


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cosine(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
