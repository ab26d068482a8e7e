"""The ablation harness (Appendix B, Table 1) on the GPU: a short run of all
eight configurations on the 32^3 masked Poisson mock of test_gpu_recon."""
import numpy as np
import pytest

from gpu_cases import table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_ablation_short_run():
    from paper_2604_26823_gb300 import build
    build.build()
    from paper_2604_26823_gb300 import ablation, api, inputs
    n, box = 32, 62.5
    lnk, lnp = table()
    R = inputs.survey_selection(n, box, 4, observer=(box / 2, box / 2, -0.3 * box), r_scale=300.0 * n / 256)
    counts = inputs.poisson_counts(0.4 * R * 1.2, 5)
    cfg = api.Config(n=n, box=box, n_steps=4, lpt_order=2, likelihood="poisson", nbar_cell=0.4, alpha=0.7,
                     delta_th=1.2, K=3.0, rho_floor=1e-3, prior_weight=1.0)
    plan = api.Plan(cfg, lnk, lnp)
    dev = lambda x: torch.tensor(np.asarray(x), dtype=torch.float32, device="cuda")
    Rd = dev(R)
    nreal = api.pm_count_positive(plan, Rd)
    fcounts = api.pm_rom_fourier_counts(plan)
    targets = lambda it: (dev(inputs.sorted_normal_targets(nreal, 7 + it)),
                          dev(inputs.sorted_normal_targets_per_bin(fcounts, 7 + it)))
    res = ablation.ablation(plan, dev(inputs.white_noise(n, 2)), dev(counts), Rd, 12, targets, rom_every=4,
                            checkpoint_every=4, warm=(1, 2), lbfgs_checkpoints=2)
    plan.close()
    runs = res["runs"]
    assert list(runs) == ["Mujica", "L-BFGS", "L-BFGS-S-1", "L-BFGS-S-2", "L-BFGS-S-3", "M01L02", "M02L02"]
    assert np.isfinite(res["zero_likelihood"])
    assert [c[0] for c in runs["Mujica"]["curve"]] == [4, 8, 12] and runs["Mujica"]["failed"] is None
    for name, r in runs.items():
        assert all(np.isfinite(c[1]) and np.isfinite(c[2]) for c in r["curve"]), name
        if r["failed"] is None:
            # every accepted L-BFGS step lowers the loss unless a matching intervened
            losses = [c[2] for c in r["curve"]]
            if name != "Mujica":
                assert all(b < a for a, b in zip(losses[:-1], losses[1:])), name
    # the smallest cap moves least from the common start in the same number of iterations
    a, b = runs["L-BFGS-S-3"], runs["L-BFGS"]
    if a["failed"] is None and b["failed"] is None:
        assert a["curve"][-1][2] >= b["curve"][-1][2]
