"""Ablation harness: MujicΛ against vanilla L-BFGS (Appendix B, Table 1).

Runs, all on one plan and one mock:
  Mujica      projected L-BFGS from s0 with rank-order matching every
              ``rom_every`` iterations, a checkpoint every ``checkpoint_every``
              iterations (right after the matching when both fall together);
  L-BFGS, L-BFGS-S-1, -S-2, -S-3
              unconstrained L-BFGS (no projection, no rank-order matching) from
              the same s0 with the line-search step capped at 1, 0.1, 0.01,
              0.001;
  MjjLkk      the same L-BFGS with cap 1 started from Mujica checkpoint #jj and
              run for kk checkpoints (the paper: M05L30, M10L30, M15L30).
Every run records the likelihood term (the negative log-likelihood; the paper
plots its negative) at each of its checkpoints.  The homogeneous solution
s = 0 gives the reference level of the paper's figure.  A vanilla run whose
line search fails (no finite Armijo point along d or along -g) stops there and
says so.

Every arithmetic step runs in the library's kernels (through ``recon``); this
module only sequences runs and collects their curves.
"""
import time

import torch

from . import api, recon


def run_names(eps_caps=(1.0, 0.1, 0.01, 0.001), warm=(5, 10, 15), lbfgs_checkpoints=30):
    """Names of the runs in Table 1's order."""
    names = ["Mujica"]
    names += ["L-BFGS" if i == 0 else f"L-BFGS-S-{i}" for i in range(len(eps_caps))]
    names += [f"M{j:02d}L{lbfgs_checkpoints:02d}" for j in warm]
    return names


def ablation(plan, s0, data, R, iters, rom_targets, rom_every=20, checkpoint_every=20,
             eps_caps=(1.0, 0.1, 0.01, 0.001), warm=(5, 10, 15), lbfgs_checkpoints=None, seed=6):
    """Run Table 1 on (plan, data, R) from s0 (device tensors of the plan's
    dtype).  ``iters`` iterations per run from s0; warm-started runs take
    ``lbfgs_checkpoints`` checkpoints (default: as many as fit in iters).
    Returns {"zero_likelihood": L(s = 0), "runs": {name: {...}}} where each run
    holds its checkpoint curve [(iteration, likelihood, loss)], final loss,
    wall time and driver counters."""
    if lbfgs_checkpoints is None:
        lbfgs_checkpoints = iters // checkpoint_every
    names = run_names(eps_caps, warm, lbfgs_checkpoints)
    out = {"runs": {}}
    g = torch.empty_like(s0)
    api.pm_adjoint(plan, torch.zeros_like(s0), data, R, grad_out=g)
    out["zero_likelihood"] = api.pm_last_terms(plan)[0]

    def run(name, start, n_iter, keep=None, **kw):
        curve = []

        def on_checkpoint(it, s, loss, lik):
            curve.append((it, lik, loss))
            if keep is not None and len(curve) in warm:
                keep[len(curve)] = s.clone()

        t0 = time.perf_counter()
        failed = None
        try:
            _, f, info = recon.reconstruct(plan, start, data, R, n_iter, seed=seed, checkpoint_every=checkpoint_every,
                                           on_checkpoint=on_checkpoint, **kw)
        except recon.LineSearchError as e:
            f, info, failed = float("nan"), {}, str(e)
        if start.is_cuda:
            torch.cuda.synchronize()
        out["runs"][name] = {"curve": curve, "final_loss": f, "seconds": time.perf_counter() - t0, "failed": failed,
                             **{k: v for k, v in info.items() if isinstance(v, (int, float))}}

    by_index = {}   # Mujica checkpoint number (from 1) -> state, for the warm starts
    run(names[0], s0, iters, keep=by_index, rom_every=rom_every, rom_targets=rom_targets, project=True)
    for name, cap in zip(names[1:1 + len(eps_caps)], eps_caps):
        run(name, s0, iters, rom_every=0, project=False, eps_max=cap)
    for name, j in zip(names[1 + len(eps_caps):], warm):
        if j not in by_index:
            out["runs"][name] = {"curve": [], "failed": f"the Mujica run has no checkpoint #{j}"}
            continue
        run(name, by_index[j], lbfgs_checkpoints * checkpoint_every, rom_every=0, project=False, eps_max=1.0)
    return out


def _main():
    import argparse
    import json

    import numpy as np

    from . import build, inputs
    ap = argparse.ArgumentParser(description="MujicΛ vs vanilla L-BFGS ablation (Table 1) on the masked mock")
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--box", type=float, default=125.0)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--checkpoint-every", type=int, default=20)
    ap.add_argument("--rom-every", type=int, default=20)
    args = ap.parse_args()
    build.build()
    lnk, lnp = api.pm_linear_power_table()
    R, s_true, counts, nbar_cell = recon.masked_mock(args.n, args.box, n_steps=args.steps, lnk=lnk, lnp=lnp)
    dev = lambda x: torch.as_tensor(np.asarray(x)).to(device="cuda", dtype=torch.float32)
    plan = api.Plan(recon.mock_config(args.n, args.box, nbar_cell, "f32", n_steps=args.steps), lnk, lnp)
    Rd = dev(R)
    nreal = api.pm_count_positive(plan, Rd)
    fcounts = api.pm_rom_fourier_counts(plan)
    targets = lambda it: (dev(inputs.sorted_normal_targets(nreal, 7 + it)),
                          dev(inputs.sorted_normal_targets_per_bin(fcounts, 7 + it)))
    res = ablation(plan, dev(inputs.white_noise(args.n, 2)), dev(counts), Rd, args.iters, targets,
                   rom_every=args.rom_every, checkpoint_every=args.checkpoint_every)
    res.update({"workload": f"ablation-masked-{args.n}", "n": args.n, "box": args.box, "iters": args.iters,
                "galaxies": float(counts.sum())})
    plan.close()
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    _main()
