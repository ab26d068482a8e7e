"""Annealing on the GPU (Sec. 3, opening): the resolution transfer of the
white noise (pm_refine_noise) and the coarsening of the data (pm_coarsen)
against the oracle, the transfer's defining property through the library's
own linear field, and a two-stage reconstruction.

Tolerances: the transfer is one forward and one inverse FFT of unit white
noise, so FP32 agrees to ~1e-7 per element (1e-5 relative L2 written) and
FP64 to ~1e-15 (1e-12 written); block sums of integer counts are exact in
both precisions (bit-exact test); block means of R in FP32 are one rounding of
an FP64 sum (1e-7 relative per element)."""
import numpy as np
import pytest

from oracle import anneal as OA
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
    return torch.tensor(np.asarray(x), dtype=_dt(prec), device="cuda")


def _plan(api, n, prec, box=64.0):
    lnk, lnp = table()
    return api.Plan(api.Config(n=n, box=box, n_steps=2, precision=prec), lnk, lnp)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("nc,n", [(16, 32), (8, 32), (2, 16), (32, 64)])
def test_refine_noise_matches_oracle(api, nc, n, prec):
    from paper_2604_26823_gb300 import inputs
    sc = inputs.white_noise(nc, 21).astype(np.float64)
    fresh = inputs.white_noise(n, 22).astype(np.float64)
    plan = _plan(api, n, prec)
    out = api.pm_refine_noise(plan, _dev(sc, prec), _dev(fresh, prec)).cpu().numpy()
    ref = OA.refine_noise(sc, fresh)
    assert rel_l2(out, ref) < (1e-5 if prec == "f32" else 1e-12)
    plan.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_refined_field_keeps_the_coarse_linear_density(api, prec):
    """With no fresh noise and a coarse field without Nyquist-plane modes, the
    fine linear density at the coarse nodes equals the coarse linear density
    (same box, same P(k)): the transfer keeps delta_L, not just s."""
    from paper_2604_26823_gb300 import inputs
    nc, n = 16, 32
    S = np.fft.fftn(inputs.white_noise(nc, 23).astype(np.float64))
    S[nc // 2], S[:, nc // 2], S[:, :, nc // 2] = 0, 0, 0
    sc = np.fft.ifftn(S).real
    pc, pf = _plan(api, nc, prec), _plan(api, n, prec)
    sf = api.pm_refine_noise(pf, _dev(sc, prec), torch.zeros((n, n, n), dtype=_dt(prec), device="cuda"))
    dc = api.pm_linear_field(pc, _dev(sc, prec)).cpu().numpy()
    df = api.pm_linear_field(pf, sf).cpu().numpy()
    assert rel_l2(df[::2, ::2, ::2], dc) < (1e-5 if prec == "f32" else 1e-12)
    pc.close()
    pf.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,f", [(32, 2), (64, 4), (16, 16)])
def test_coarsen_matches_oracle(api, n, f, prec):
    from paper_2604_26823_gb300 import inputs
    counts = inputs.poisson_counts(np.full((n, n, n), 0.7), 24).astype(np.float64)
    R = inputs.uniform_field(n, 25, 0.0, 1.0).astype(np.float64)
    got = api.pm_coarsen(_dev(counts, prec), f).cpu().numpy()
    np.testing.assert_array_equal(got, OA.coarsen(counts, f))
    gm = api.pm_coarsen(_dev(R, prec), f, mean=True).cpu().numpy().astype(np.float64)
    rm = OA.coarsen(R.astype(np.float32) if prec == "f32" else R, f, mean=True)
    np.testing.assert_allclose(gm, rm, rtol=1e-7 if prec == "f32" else 1e-15, atol=0)


def test_refine_noise_rejects_bad_sizes(api):
    from paper_2604_26823_gb300 import _lib as L
    plan = _plan(api, 32, "f32")
    z = lambda k: torch.zeros((k, k, k), dtype=torch.float32, device="cuda")
    for nc in (32, 12):
        with pytest.raises(RuntimeError):
            L.check(L.load().pm_refine_noise(plan.handle, api._ptr(z(nc), torch.float32, nc ** 3, "s"), nc,
                                             plan.mesh(z(32), "f"), plan.mesh(z(32), "o"), None), "refine")
    plan.close()


def test_annealed_reconstruction(api):
    """Two stages on a masked Poisson mock (16^3 then 32^3 in 62.5 Mpc/h),
    with rank-order matching every 5 (coarse) and 3 (fine) iterations."""
    from paper_2604_26823_gb300 import inputs, recon
    n, box, f = 32, 62.5, 2
    lnk, lnp = table()
    R = inputs.survey_selection(n, box, 4, observer=(box / 2, box / 2, -0.3 * box), r_scale=300.0 * n / 256)
    counts = inputs.poisson_counts(0.4 * R * 1.2, 5)
    cfg = api.Config(n=n, box=box, n_steps=4, lpt_order=2, likelihood="poisson", nbar_cell=0.4, alpha=0.7,
                     delta_th=1.2, K=3.0, rho_floor=1e-3, prior_weight=1.0)
    dev = lambda x: torch.tensor(np.asarray(x), dtype=torch.float32, device="cuda")

    def targets_for(plan, Rm):
        nreal = api.pm_count_positive(plan, Rm)
        fcounts = api.pm_rom_fourier_counts(plan)
        return lambda it: (dev(inputs.sorted_normal_targets(nreal, 7 + it)),
                           dev(inputs.sorted_normal_targets_per_bin(fcounts, 7 + it)))

    trace = []
    s, loss, info = recon.anneal(cfg, lnk, lnp, dev(inputs.white_noise(n // f, 2)), dev(counts), dev(R), f,
                                 iters_coarse=8, iters_fine=6, fresh=dev(inputs.white_noise(n, 8)),
                                 rom_every_coarse=5, rom_every_fine=3, targets_for=targets_for, trace=trace)
    assert np.isfinite(loss) and s.shape == (n, n, n)
    coarse, fine = trace[:9], trace[9:]
    assert [i for i, _ in coarse] == list(range(9)) and [i for i, _ in fine] == list(range(7))
    # before its first rank-order matching each stage lowers its loss step by
    # step (Armijo); a matching may raise it, and every step after one lowers
    # it again
    assert coarse[4][1] < coarse[0][1] and fine[2][1] < fine[0][1]
    for tr, rom in ((coarse, 5), (fine, 3)):
        for (i0, l0), (i1, l1) in zip(tr[:-1], tr[1:]):
            if i1 % rom:
                assert l1 < l0
    assert info["coarse"]["rom"] == 1 and info["fine"]["rom"] == 2
