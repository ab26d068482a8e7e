"""The benchmark configuration at full size (256^3, 10 steps, masked Poisson
likelihood, the launch configuration bench.py times), checked through
properties that hold at any size -- the FP64 oracle cannot evaluate a 256^3
gradient in test time:
  * FP32 path vs the all-FP64 GPU path: loss and density within 1e-5, the
    gradient's cosine >= 0.99999 and its relative L2 within 1.5 x the
    largest error of two FP64 evaluations from inputs perturbed so that their
    trajectory deviates by the FP32 path's own final-displacement error (the
    FP32 error is set by the few particles whose CIC derivative branch flips,
    a random quantity: measured 3.4e-4 .. 8.5e-4 over four seeds, and
    2.8e-4 .. 1.9e-3 for such perturbed FP64 evaluations);
  * the FP64 path's gradient against its own central differences along
    seeded random directions (eps = 1e-3);
  * bit-identical repeated evaluation, and bit-identical gradients with
    particle-state checkpointing every 2 steps.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 256


@pytest.fixture(scope="module")
def setup():
    import bench
    from paper_2604_26823_gb300 import build
    build.build()
    from paper_2604_26823_gb300 import api, inputs, recon
    lnk, lnp = api.pm_linear_power_table()
    R, s_true, counts, nbar_cell = recon.masked_mock(N, bench.BOX, n_steps=bench.STEPS_PM, nbar=bench.NBAR,
                                                    lnk=lnk, lnp=lnp)
    plan32 = api.Plan(bench.config(api, nbar_cell, "f32"), lnk, lnp)
    s0 = inputs.white_noise(N, 2)
    return dict(api=api, bench=bench, lnk=lnk, lnp=lnp, R=R, counts=counts, s0=s0, nbar=nbar_cell,
                plan32=plan32)


def _eval(api, plan, s, counts, R, dtype):
    d = lambda x: torch.tensor(x, dtype=dtype, device="cuda")
    delta = torch.empty((N, N, N), dtype=dtype, device="cuda")
    loss = api.pm_forward(plan, d(s), d(counts), d(R), delta_out=delta)
    l2, g = api.pm_adjoint(plan, d(s), d(counts), d(R))
    assert l2 == loss
    return loss, delta.double().cpu().numpy(), g.double().cpu().numpy()


def test_fp32_vs_fp64_at_full_size(setup):
    api, bench = setup["api"], setup["bench"]
    l32, d32, g32 = _eval(api, setup["plan32"], setup["s0"], setup["counts"], setup["R"], torch.float32)
    plan64 = api.Plan(bench.config(api, setup["nbar"], "f64"), setup["lnk"], setup["lnp"])
    l64, d64, g64 = _eval(api, plan64, setup["s0"], setup["counts"], setup["R"], torch.float64)
    del plan64
    assert abs(l32 - l64) < 1e-5 * abs(l64)
    assert np.linalg.norm(d32 - d64) / np.linalg.norm(d64) < 1e-5
    cos = float(g32.ravel() @ g64.ravel() / (np.linalg.norm(g32) * np.linalg.norm(g64)))
    err = np.linalg.norm(g32 - g64) / np.linalg.norm(g64)
    print(f"256^3 FP32 vs FP64 path: loss {abs(l32 - l64) / abs(l64):.2e}, density "
          f"{np.linalg.norm(d32 - d64) / np.linalg.norm(d64):.2e}, gradient rel L2 {err:.3e} cos {cos:.9f}")
    assert cos > 0.99999
    # the FP32-level error of this seed: FP64 evaluations whose trajectory
    # deviates by the FP32 path's own final-displacement error
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    dd = lambda x, dt: torch.tensor(x, dtype=dt, device="cuda")
    plan64 = api.Plan(bench.config(api, setup["nbar"], "f64"), setup["lnk"], setup["lnp"])
    s0 = setup["s0"].astype(np.float64)
    x64 = api.pm_evolve(plan64, dd(s0, torch.float64))[0].cpu().numpy()
    x32 = api.pm_evolve(setup["plan32"], dd(s0, torch.float32))[0].double().cpu().numpy()
    traj = rel(x32, x64)
    levels = []
    for k in range(2):
        xi = np.random.default_rng(200 + k).standard_normal(s0.shape)
        e0 = rel(api.pm_evolve(plan64, dd(s0 + 1e-6 * xi, torch.float64))[0].cpu().numpy(), x64)
        amp = 1e-6 * traj / e0
        _, _, gp = _eval(api, plan64, s0 + amp * xi, setup["counts"], setup["R"], torch.float64)
        levels.append(rel(gp, g64))
    del plan64
    bound = 1.5 * max(max(levels), 1e-4)
    print(f"256^3 FP32 final displacement rel L2 {traj:.3e}; trajectory-matched FP64 evaluations: "
          + ", ".join(f"{v:.3e}" for v in levels) + f"; bound {bound:.3e}")
    assert err < bound, (err, bound)


def test_fp64_gradient_against_finite_differences(setup):
    api, bench = setup["api"], setup["bench"]
    from paper_2604_26823_gb300 import inputs
    plan64 = api.Plan(bench.config(api, setup["nbar"], "f64"), setup["lnk"], setup["lnp"])
    d = lambda x: torch.tensor(x, dtype=torch.float64, device="cuda")
    s, c, R = d(setup["s0"]), d(setup["counts"]), d(setup["R"])
    _, g = api.pm_adjoint(plan64, s, c, R)
    errs = []
    for u in inputs.random_unit_directions(N, 4, 100):
        u = d(u)
        fd = (api.pm_forward(plan64, s + 1e-3 * u, c, R) - api.pm_forward(plan64, s - 1e-3 * u, c, R)) / 2e-3
        gu = float((g * u).sum())
        errs.append(abs(fd - gu) / (abs(gu) + 1e-3 * float(g.norm())))
    del plan64
    print("256^3 FP64 gradient vs FD along 4 directions:", ["%.2e" % e for e in errs])
    assert max(errs) < 5e-4, errs   # measured 1.9e-4 at worst (eps = 1e-3 crosses cell faces)


def test_repeatable_and_checkpoint_identical(setup):
    api, bench = setup["api"], setup["bench"]
    d = lambda x: torch.tensor(x, dtype=torch.float32, device="cuda")
    s, c, R = d(setup["s0"]), d(setup["counts"]), d(setup["R"])
    la, ga = api.pm_adjoint(setup["plan32"], s, c, R)
    lb, gb = api.pm_adjoint(setup["plan32"], s, c, R)
    assert la == lb and torch.equal(ga, gb)
    cfg = bench.config(api, setup["nbar"], "f32")
    cfg.checkpoint_every = 2
    plan_ck = api.Plan(cfg, setup["lnk"], setup["lnp"])
    lc, gc = api.pm_adjoint(plan_ck, s, c, R)
    assert lc == la and torch.equal(gc, ga)
