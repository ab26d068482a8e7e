"""Host logic of the reconstruction driver's ablation options and of the
ablation harness (Appendix B, Table 1), run on the CPU against a fake of the
library calls: a quadratic loss (likelihood 1/2 sum a (s - t)^2 plus the prior
1/2 sum s^2), the oracle's L-BFGS two-loop recursion, and a projection /
rank-order matching that records its calls and leaves s unchanged."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lbfgs as OL
from paper_2604_26823_gb300 import ablation, recon


class FakePlan:
    dtype = torch.float64

    def __init__(self, a, t):
        self.a, self.t = a, t
        self.terms = (0.0, 0.0)


class FakeApi:
    """The library calls the driver makes, on CPU tensors."""

    def __init__(self):
        self.calls = []          # (kind, mode, step length or evaluated s)

    class LBFGS:
        def __init__(self, n, m=10, precision="f64"):
            self.o = OL.LBFGS(m)

        def close(self):
            pass

    def lbfgs_step(self, st, s, g):
        d, gd, pushed = st.o.step(s.numpy(), g.numpy())
        d = torch.tensor(d).reshape(s.shape)
        return d, gd, float(d.norm()), pushed

    def lbfgs_reset(self, st):
        st.o.reset()
        st.o.x_prev = st.o.g_prev = None

    def pm_axpy(self, alpha, x, y, out):
        self.calls.append(("step", abs(alpha) * float(x.norm())))
        out.copy_(y + alpha * x)
        return out

    def project_rank_match(self, plan, s, mode, **kw):
        self.calls.append(("project", mode))
        return 0

    def pm_adjoint(self, plan, s, data, R, grad_out):
        lik = 0.5 * float(torch.sum(plan.a * (s - plan.t) ** 2))
        prior = 0.5 * float(torch.sum(s * s))
        grad_out.copy_(plan.a * (s - plan.t) + s)
        plan.terms = (lik, prior)
        self.calls.append(("eval", s.clone()))
        return lik + prior, grad_out

    def pm_last_terms(self, plan):
        return plan.terms


@pytest.fixture()
def fake(monkeypatch):
    f = FakeApi()
    monkeypatch.setattr(recon, "api", f)
    monkeypatch.setattr(ablation, "api", f)
    rng = np.random.default_rng(3)
    n = 6
    plan = FakePlan(torch.tensor(rng.uniform(0.5, 4.0, (n, n, n))), torch.tensor(rng.normal(0, 1, (n, n, n))))
    s0 = torch.tensor(rng.normal(0, 1, (n, n, n)))
    targets = lambda it: (None, None)
    return f, plan, s0, targets


def test_table1_run_names():
    assert ablation.run_names() == ["Mujica", "L-BFGS", "L-BFGS-S-1", "L-BFGS-S-2", "L-BFGS-S-3",
                                    "M05L30", "M10L30", "M15L30"]


def test_vanilla_options_and_checkpoints(fake):
    f, plan, s0, targets = fake
    seen = []
    s, loss, info = recon.reconstruct(plan, s0, None, None, 12, rom_every=0, project=False, eps_max=0.01,
                                      checkpoint_every=4, on_checkpoint=lambda it, s, l, lik: seen.append((it, l, lik)))
    assert not [c for c in f.calls if c[0] == "project"]
    steps = [c[1] for c in f.calls if c[0] == "step"]
    assert max(steps) <= 0.01 + 1e-15                     # every trial step capped at eps_max
    assert [it for it, _, _ in seen] == [4, 8, 12]
    assert all(lik < l for _, l, lik in seen)             # likelihood term = loss minus the prior
    assert info["rom"] == 0 and np.isfinite(loss)


def test_projected_driver_projects_every_trial_and_matches(fake):
    f, plan, s0, targets = fake
    recon.reconstruct(plan, s0, None, None, 10, rom_every=5, rom_targets=targets, project=True)
    modes = [c[1] for c in f.calls if c[0] == "project"]
    trials = len([c for c in f.calls if c[0] == "step"])
    assert modes.count(1) == trials                       # PM_PROJECT alone on each trial point
    assert modes.count(7) == 2                            # Fourier + real ROM + projection at 5 and 10


def test_ablation_harness(fake):
    f, plan, s0, targets = fake
    res = ablation.ablation(plan, s0, None, None, 12, targets, rom_every=4, checkpoint_every=4, warm=(1, 2, 5),
                            lbfgs_checkpoints=2)
    runs = res["runs"]
    assert list(runs) == ["Mujica", "L-BFGS", "L-BFGS-S-1", "L-BFGS-S-2", "L-BFGS-S-3", "M01L02", "M02L02",
                          "M05L02"]
    assert res["zero_likelihood"] == pytest.approx(0.5 * float(torch.sum(plan.a * plan.t ** 2)))
    assert [c[0] for c in runs["Mujica"]["curve"]] == [4, 8, 12]
    for name in ("L-BFGS", "L-BFGS-S-1", "L-BFGS-S-2", "L-BFGS-S-3"):
        assert [c[0] for c in runs[name]["curve"]] == [4, 8, 12] and runs[name]["failed"] is None
    assert [c[0] for c in runs["M01L02"]["curve"]] == [4, 8]
    assert runs["M05L02"]["failed"] and runs["M05L02"]["curve"] == []   # the baseline has 3 checkpoints
    # smaller caps make less progress on the quadratic after the same number of iterations
    fin = [runs[n]["curve"][-1][2] for n in ("L-BFGS", "L-BFGS-S-1", "L-BFGS-S-2", "L-BFGS-S-3")]
    assert fin[0] <= fin[1] <= fin[2] <= fin[3]


def test_nonfinite_trial_is_rejected(fake, monkeypatch):
    """A trial whose loss the library reports as non-finite is halved like a
    failed Armijo test, not raised."""
    from paper_2604_26823_gb300 import _lib as L
    f, plan, s0, targets = fake
    real = f.pm_adjoint
    state = {"evals": 0}

    def flaky(plan_, s, data, R, grad_out):
        state["evals"] += 1
        if state["evals"] == 2:                      # the first trial of the first iteration
            raise L.PMError(L.PM_ERR_NONFINITE, "pm_adjoint", "loss is not finite")
        return real(plan_, s, data, R, grad_out)

    monkeypatch.setattr(f, "pm_adjoint", flaky)
    _, loss, info = recon.reconstruct(plan, s0, None, None, 3, rom_every=0, project=False)
    assert np.isfinite(loss) and info["halvings"] >= 1
