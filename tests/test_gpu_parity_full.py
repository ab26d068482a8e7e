"""Oracle parity of the kernel instances the benchmark runs, at full size.

Every mesh size is its own template instance (radix plans, tiles, launch
shapes and the >48 KB shared-memory launch path differ between 128^3, 256^3
and 512^3), so the 256^3 instances the benchmark times -- and the 512^3 ones
of the large-mesh configuration -- are compared here with the FP64 oracle
element by element:
  * linear field, 2LPT displacement and momentum, PM force and painted
    density at 256^3 (500 Mpc/h, the benchmark's cell size), FP32 and FP64;
  * linear field and density at 512^3 (1000 Mpc/h), FP32, with the force
    checked on a seeded sample of 2^20 particles the oracle reads out one by
    one (the oracle's full 512^3 readout would dominate the test's time);
  * real-space rank-order matching, bit for bit, on more than 2^20 keys (the
    radix sort's row scan then runs more than one pass);
  * lbfgs_step with the benchmark's m = 10 on 256^3 elements, past a full
    history and through a rejected pair;
  * the FP32 path's dot product g.d on 256^3 elements against the exactly
    rounded FP64 sum.
Tolerances: the FP32 path's 1e-5 relative L2 (1e-6 for the linear field, a
single FFT pair), the FP64 path's 1e-9 (1e-10 for the linear field).
"""
import math

import numpy as np
import pytest

from oracle import lbfgs as OL
from oracle import mesh as OMesh
from oracle import model as OM
from oracle import projection as OP
from gpu_cases import rel_l2, table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-9}


@pytest.fixture(scope="module")
def api():
    from paper_2604_26823_gb300 import build
    build.build()
    from paper_2604_26823_gb300 import api as A
    return A


_PLANS = {}


def plan_for(api, n, box, prec):
    key = (n, box, prec)
    if key not in _PLANS:
        # keep one full-size plan at a time (each holds several GB)
        for k in list(_PLANS):
            _PLANS.pop(k).close()
        torch.cuda.empty_cache()
        lnk, lnp = table()
        _PLANS[key] = api.Plan(api.Config(n=n, box=box, n_steps=1, precision=prec), lnk, lnp)
    return _PLANS[key]


def dev(x, prec):
    return torch.tensor(np.asarray(x), dtype=torch.float32 if prec == "f32" else torch.float64, device="cuda")


def seeded_disp(n, box, seed=7):
    """Displacements of 1.5 cells rms, representable in FP32 (both sides see
    the same values)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 1.5 * box / n, (3, n ** 3)).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_linear_field_256(api, prec):
    from paper_2604_26823_gb300 import inputs
    n, box = 256, 500.0
    plan = plan_for(api, n, box, prec)
    s = inputs.white_noise(n, 2).astype(np.float64)
    got = api.pm_linear_field(plan, dev(s, prec)).cpu().numpy()
    lnk, lnp = table()
    ref = OM.linear_field(s, OM.Config(n=n, box=box), lnk, lnp)
    err = rel_l2(got, ref)
    print(f"linear field 256^3 {prec}: rel L2 {err:.2e}")
    assert err < 0.1 * TOL[prec]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_lpt_256(api, prec):
    from paper_2604_26823_gb300 import inputs
    n, box = 256, 500.0
    plan = plan_for(api, n, box, prec)
    s = inputs.white_noise(n, 2).astype(np.float64)
    disp, mom = api.pm_lpt(plan, dev(s, prec))
    disp, mom = disp.cpu().numpy(), mom.cpu().numpy()
    lnk, lnp = table()
    rd, rm, _ = OM.lpt(s, OM.Config(n=n, box=box), lnk, lnp)
    ed, em = rel_l2(disp, rd.T), rel_l2(mom, rm.T)
    print(f"2LPT 256^3 {prec}: displacement rel L2 {ed:.2e}, momentum {em:.2e}")
    assert ed < TOL[prec] and em < TOL[prec]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_force_and_density_256(api, prec):
    n, box = 256, 500.0
    plan = plan_for(api, n, box, prec)
    disp = seeded_disp(n, box)
    f, dens = api.pm_force(plan, dev(disp, prec), with_density=True)
    f, dens = f.cpu().numpy(), dens.cpu().numpy()
    cfg = OM.Config(n=n, box=box)
    lnk, lnp = table()
    rf, _, rdelta = OM.force(disp.T, cfg, OM._Ops(cfg, lnk, lnp))
    ed, ef = rel_l2(dens, rdelta), rel_l2(f, rf.T)
    print(f"force 256^3 {prec}: density rel L2 {ed:.2e}, force {ef:.2e}")
    assert ed < TOL[prec] and ef < TOL[prec]
    # momentum conservation of the FP32 kernels at full size
    fs = np.abs(f.astype(np.float64).sum(axis=1))
    assert np.all(fs < 1e-4 * np.abs(f).astype(np.float64).sum(axis=1))


def test_linear_field_512(api):
    from paper_2604_26823_gb300 import inputs
    n, box = 512, 1000.0
    plan = plan_for(api, n, box, "f32")
    s = inputs.white_noise(n, 1).astype(np.float64)
    got = api.pm_linear_field(plan, dev(s, "f32")).cpu().numpy()
    lnk, lnp = table()
    ref = OM.linear_field(s, OM.Config(n=n, box=box), lnk, lnp)
    err = rel_l2(got, ref)
    print(f"linear field 512^3 f32: rel L2 {err:.2e}")
    assert err < 0.1 * TOL["f32"]


def test_force_and_density_512(api):
    n, box = 512, 1000.0
    plan = plan_for(api, n, box, "f32")
    disp = seeded_disp(n, box, seed=8)
    f, dens = api.pm_force(plan, dev(disp, "f32"), with_density=True)
    f, dens = f.cpu().numpy(), dens.cpu().numpy()
    cfg = OM.Config(n=n, box=box)
    lnk, lnp = table()
    ops = OM._Ops(cfg, lnk, lnp)
    # the oracle's force, step by step (paint, spectral force, readout), with
    # the readout taken at a seeded sample of particles
    u = OM.positions_cells(disp.T, cfg)
    del disp
    rdelta = OMesh.cic_paint(u, n) - 1.0
    ed = rel_l2(dens, rdelta)
    dk = OMesh.rfft3(rdelta)
    del rdelta, dens
    idx = np.sort(np.random.default_rng(9).choice(n ** 3, 1 << 20, replace=False))
    us = u[idx]
    del u
    rf = np.stack([OMesh.cic_readout(us, OMesh.irfft3(ops.force[i] * dk, n)) for i in range(3)])
    ef = rel_l2(f[:, idx], rf)
    print(f"force 512^3 f32: density rel L2 {ed:.2e}, force on 2^20 sampled particles {ef:.2e}")
    assert ed < TOL["f32"] and ef < TOL["f32"]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_real_rom_bit_exact_over_2_20_keys(api, prec):
    from paper_2604_26823_gb300 import inputs
    n = 128
    plan = plan_for(api, n, 400.0, prec)
    s = inputs.white_noise(n, 2)
    s.reshape(-1)[1000:3000] = 0.5      # ties, broken by index
    s.reshape(-1)[5000] = -0.0
    s.reshape(-1)[5001] = 0.0
    resp = inputs.uniform_field(n, 3, -0.2, 1.0)
    cnt = api.pm_count_positive(plan, dev(resp, prec))
    assert cnt == int((resp > 0).sum()) and cnt > (1 << 20)
    t = inputs.sorted_normal_targets(cnt, 4)
    x = dev(s, prec)
    rank = torch.zeros(n ** 3, dtype=torch.int32, device="cuda")
    api.project_rank_match(plan, x, api.L.PM_ROM_REAL, R=dev(resp, prec), targets_real=dev(t, prec), rank_out=rank)
    ref = OP.rom_real(s.astype(np.float64), resp.astype(np.float64), t.astype(np.float64))
    np.testing.assert_array_equal(x.cpu().numpy().astype(np.float64), ref)
    np.testing.assert_array_equal(rank.cpu().numpy().astype(np.int64),
                                  OP.rom_real_ranks(s.astype(np.float64), resp).reshape(-1))


def _q(x, prec):
    return x.astype(np.float32).astype(np.float64) if prec == "f32" else x


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_lbfgs_256_m10_full_history_and_rejected_pair(api, prec):
    """15 steps of a convex quadratic (12 pairs pushed, so the ring of 10 has
    wrapped), one step whose pair fails the curvature test (y = -s) with the
    history full, then two more steps: every direction, g.d and |d| match the
    oracle, which stores only accepted pairs."""
    n, m = 256 ** 3, 10
    rng = np.random.default_rng(3)
    a = rng.uniform(0.5, 3.0, n)
    b = rng.standard_normal(n)
    st = api.LBFGS(n, m=m, precision=prec)
    ref = OL.LBFGS(m=m)
    x = np.zeros(n)
    g_prev = x_prev = None
    tol_d = 1e-5 if prec == "f32" else 1e-11
    tol_s = 1e-6 if prec == "f32" else 1e-11
    pushes = 0
    for it in range(18):
        xq = _q(x, prec)
        if it == 15:
            g = g_prev - 0.5 * (xq - x_prev)    # y = -s / 2: s.y < 0, rejected
        else:
            g = a * xq - b
        gq = _q(g, prec)
        d, gd, dn, pushed = api.lbfgs_step(st, dev(xq, prec), dev(gq, prec))
        rd, rgd, rpushed = ref.step(xq, gq)
        assert pushed == rpushed, it
        pushes += int(pushed)
        if it == 15:
            assert not pushed and len(ref.s) == m
        d = d.cpu().numpy().astype(np.float64)
        ed = rel_l2(d, rd)
        assert ed < tol_d, (it, ed)
        assert abs(gd - rgd) < tol_s * abs(rgd), (it, gd, rgd)
        assert abs(dn - np.linalg.norm(rd)) < tol_s * np.linalg.norm(rd), it
        x_prev, g_prev = xq, gq
        x = xq + 0.5 * rd / max(1.0, np.linalg.norm(rd))
    assert pushes >= 12


def test_fp32_dot_against_exact_sum(api):
    """g.d of the FP32 path (exact products, compensated FP32 sums per
    thread, FP64 across threads) on 256^3 elements against the correctly
    rounded sum of the exact products (math.fsum): relative error <= 1e-12."""
    n = 256 ** 3
    rng = np.random.default_rng(5)
    st = api.LBFGS(n, m=10, precision="f32")
    x0 = rng.standard_normal(n).astype(np.float32)
    g0 = (rng.standard_normal(n) * np.exp(rng.uniform(-8, 8, n))).astype(np.float32)
    # first call: no pair, d = -g, g.d = -|g|^2
    d, gd, dn, _ = api.lbfgs_step(st, dev(x0, "f32"), dev(g0, "f32"))
    g64 = g0.astype(np.float64)
    exact = -math.fsum(g64 * g64)
    assert abs(gd - exact) <= 1e-12 * abs(exact), (gd, exact)
    assert abs(dn - math.sqrt(-exact)) <= 1e-12 * math.sqrt(-exact)
    # second call: one pair, d from the two-loop recursion; g.d against the
    # exact sum of the FP32 vectors' products (each exact in FP64)
    x1 = (x0 + 0.01 * rng.standard_normal(n)).astype(np.float32)
    g1 = (g0 + 0.3 * (x1.astype(np.float64) - x0)).astype(np.float32)
    d, gd, dn, pushed = api.lbfgs_step(st, dev(x1, "f32"), dev(g1, "f32"))
    assert pushed
    dd = d.cpu().numpy().astype(np.float64)
    exact = math.fsum(g1.astype(np.float64) * dd)
    assert abs(gd - exact) <= 1e-12 * abs(exact), (gd, exact)
    assert abs(dn - math.sqrt(math.fsum(dd * dd))) <= 1e-12 * dn
