"""Augmented L-BFGS reconstruction of the initial white noise (Sec. 2.3-2.4).

Each iteration:
  1. ``lbfgs_step`` pushes the pair from the previous accepted point and
     returns d = -H g (two-loop recursion, FP64 dots);
  2. projected backtracking line search along p_hat = d / |d|: trial
     s' = P(s + eps p_hat) with eps_0 = min(|d|, eps_max), Armijo test
     f(s') <= f + c1 eps g.p_hat, eps halved up to ``max_halvings`` times.
     Trials are evaluated with ``pm_adjoint`` so the accepted trial already
     carries its gradient (the first trial is accepted in the usual case).
     On failure the history is cleared and the search is repeated along -g;
     a second failure raises ``LineSearchError``;
  3. every ``rom_every`` iterations: Fourier then real-space rank-order
     matching and the projection (``project_rank_match``), then f and g are
     recomputed and the L-BFGS history is cleared.
P is the projection of Sec. 2.3.1 (z-score, |s| > 10 reset from a
counter-based normal stream keyed by (seed, counter, index)); the counter
advances by one per projection call.

Every arithmetic step runs in the library's kernels; this module only
sequences the C-ABI calls.  ``masked_mock`` builds the masked Poisson mock
of the benchmark workload with the library's own forward model.
"""
import math
import time

import numpy as np
import torch

from . import _lib as L
from . import api, inputs


class LineSearchError(RuntimeError):
    pass


def reconstruct(plan, s0, data, R, iters, m=10, eps_max=1.0, c1=1e-4, max_halvings=30, rom_every=20,
                rom_targets=None, seed=6, trace=None, project=True, checkpoint_every=0, on_checkpoint=None):
    """Run ``iters`` iterations from s0 (not modified).

    rom_targets(it) -> (targets_real, targets_fourier), device tensors of the
    plan's dtype, sorted descending (required when rom_every > 0).
    trace: optional list receiving (iteration, loss) after every iteration.
    project=False with rom_every=0 is the vanilla L-BFGS of the ablation
    (Appendix B): no projection of the trial points, no rank-order matching.
    checkpoint_every > 0: after every that many iterations (after the
    rank-order matching when both fall on the iteration) ``on_checkpoint``
    is called with (iteration, s, loss, likelihood term); s is the driver's
    own buffer, to be copied if kept.
    Returns (s, loss, info)."""
    if rom_every and rom_targets is None:
        raise ValueError("rom_every > 0 needs rom_targets")
    prec = "f64" if plan.dtype == torch.float64 else "f32"
    st = api.LBFGS(s0.numel(), m=m, precision=prec)
    s = s0.clone()
    trial = torch.empty_like(s)
    g = torch.empty_like(s)
    gt = torch.empty_like(s)
    f, _ = api.pm_adjoint(plan, s, data, R, grad_out=g)
    info = {"evals": 1, "halvings": 0, "direction_resets": 0, "rom": 0, "resets_of_values": 0}
    counter = 0
    if trace is not None:
        trace.append((0, f))
    for it in range(1, iters + 1):
        d, gd, dn, _ = api.lbfgs_step(st, s, g)
        accepted = False
        for attempt in range(2):
            eps = min(dn, eps_max)
            slope = gd / dn
            for t in range(max_halvings + 1):
                api.pm_axpy(eps / dn, d, s, out=trial)
                if project:
                    info["resets_of_values"] += api.project_rank_match(plan, trial, L.PM_PROJECT, seed=seed,
                                                                       counter=counter)
                    counter += 1
                try:
                    ft, _ = api.pm_adjoint(plan, trial, data, R, grad_out=gt)
                except L.PMError as e:   # a trial with a non-finite loss is rejected like any other
                    if e.status != L.PM_ERR_NONFINITE:
                        raise
                    ft = math.inf
                info["evals"] += 1
                if math.isfinite(ft) and ft <= f + c1 * eps * slope:
                    accepted = True
                    info["halvings"] += t
                    break
                eps *= 0.5
            if accepted:
                break
            if attempt == 0:
                api.lbfgs_reset(st)
                d, gd, dn, _ = api.lbfgs_step(st, s, g)  # empty history: d = -g
                info["direction_resets"] += 1
        if not accepted:
            raise LineSearchError(f"line search failed at iteration {it} (f = {f})")
        s, trial = trial, s
        g, gt = gt, g
        f = ft
        if rom_every and it % rom_every == 0:
            tr, tf = rom_targets(it)
            mode = L.PM_ROM_FOURIER | L.PM_ROM_REAL | L.PM_PROJECT
            api.project_rank_match(plan, s, mode, R=R, targets_real=tr, targets_fourier=tf, seed=seed,
                                   counter=counter)
            counter += 1
            f, _ = api.pm_adjoint(plan, s, data, R, grad_out=g)
            info["evals"] += 1
            info["rom"] += 1
            api.lbfgs_reset(st)
        if checkpoint_every and it % checkpoint_every == 0 and on_checkpoint is not None:
            on_checkpoint(it, s, f, api.pm_last_terms(plan)[0])
        if trace is not None:
            trace.append((it, f))
    st.close()
    return s, f, info


def anneal(cfg, lnk, lnp, s0_coarse, data, R, factor, iters_coarse, iters_fine, fresh, rom_every_coarse=5,
           rom_every_fine=20, targets_for=None, seed=6, trace=None):
    """Annealed reconstruction (Sec. 3, opening): ``iters_coarse`` iterations at
    n / factor cells per side (same box; counts summed and R averaged over each
    factor^3 block by ``pm_coarsen``; nbar_cell scaled by factor^3), then the
    coarse result carried to the fine mesh by ``pm_refine_noise`` (coarse
    modes kept, ``fresh`` on the others) and ``iters_fine`` iterations there.

    cfg: the fine ``api.Config``; s0_coarse [n_c^3], data / R / fresh [n^3]:
    device tensors of cfg's dtype.  targets_for(plan, R)(it) -> ROM targets
    as ``reconstruct`` takes them (needed when a rom_every is > 0).
    Returns (s, loss, info) with per-stage info and wall times."""
    import dataclasses
    nc = cfg.n // factor
    cfg_c = dataclasses.replace(cfg, n=nc, nbar_cell=cfg.nbar_cell * factor ** 3)
    data_c = api.pm_coarsen(data, factor)
    R_c = api.pm_coarsen(R, factor, mean=True)
    info = {}
    plan_c = api.Plan(cfg_c, lnk, lnp)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tg = targets_for(plan_c, R_c) if targets_for and rom_every_coarse else None
        s_c, f_c, info["coarse"] = reconstruct(plan_c, s0_coarse, data_c, R_c, iters_coarse, rom_every=rom_every_coarse,
                                               rom_targets=tg, seed=seed, trace=trace)
        torch.cuda.synchronize()
        info["coarse"]["seconds"] = time.perf_counter() - t0
        info["coarse"]["final_loss"] = f_c
    finally:
        plan_c.close()
    plan = api.Plan(cfg, lnk, lnp)
    try:
        t0 = time.perf_counter()
        s1 = api.pm_refine_noise(plan, s_c, fresh)
        tg = targets_for(plan, R) if targets_for and rom_every_fine else None
        s, f, info["fine"] = reconstruct(plan, s1, data, R, iters_fine, rom_every=rom_every_fine, rom_targets=tg,
                                         seed=seed, trace=trace)
        torch.cuda.synchronize()
        info["fine"]["seconds"] = time.perf_counter() - t0
    finally:
        plan.close()
    return s, f, info


def masked_mock(n, box, n_steps=10, nbar=1e-3, seed_truth=1, seed_counts=3, seed_holes=4, lnk=None, lnp=None):
    """Masked Poisson mock of the benchmark workload: selection R (40 deg cone,
    radial n(r), angular holes), s_true, the mean-density normalisation
    nbar_cell = nbar Delta^3 / mean_box[(1+delta)^alpha sigmoid(K(delta-delta_th))]
    and counts N_G ~ Poisson(R lambda(s_true)).  Returns host arrays
    (R, s_true, counts) and nbar_cell."""
    if lnk is None:
        lnk, lnp = api.pm_linear_power_table()
    dev = lambda x: torch.tensor(x, dtype=torch.float32, device="cuda")
    R = inputs.survey_selection(n, box, seed=seed_holes)
    s_true = inputs.white_noise(n, seed_truth)
    probe = api.Plan(mock_config(n, box, 1.0, n_steps=n_steps), lnk, lnp)
    ones = dev(np.ones((n, n, n), np.float32))
    gsel = api.pm_expected_counts(probe, dev(s_true), ones)
    mean_g = float(gsel.cpu().numpy().astype(np.float64).mean())
    del gsel, ones
    nbar_cell = nbar * (box / n) ** 3 / mean_g
    probe.close()
    plan = api.Plan(mock_config(n, box, nbar_cell, n_steps=n_steps), lnk, lnp)
    lam = api.pm_expected_counts(plan, dev(s_true), dev(R))
    counts = inputs.poisson_counts(lam.cpu().numpy(), seed_counts)
    plan.close()
    del lam
    torch.cuda.empty_cache()
    return R, s_true, counts, nbar_cell


def mock_config(n, box, nbar_cell, precision="f32", n_steps=10):
    """Masked Poisson configuration: 2LPT to a = 0.1, n_steps KDK steps, power-law
    + sigmoid bias (alpha, delta_th, K) = (0.7, 1.2, 3.0), rho floor 1e-3, prior on."""
    return api.Config(n=n, box=box, n_steps=n_steps, lpt_order=2, rsd_axis=-1, likelihood="poisson",
                      precision=precision, alpha=0.7, delta_th=1.2, K=3.0, nbar_cell=nbar_cell, rho_floor=1e-3,
                      prior_weight=1.0)


def cross_correlation(a, b, box, n_bins=16):
    """r(k) = P_ab / sqrt(P_aa P_bb) in |k| shells (host numpy; analysis of
    a result, not part of the hot path).  Returns (k centres, r)."""
    n = a.shape[0]
    fa, fb = np.fft.rfftn(a.astype(np.float64)), np.fft.rfftn(b.astype(np.float64))
    kf = 2 * np.pi / box
    kx = np.fft.fftfreq(n, 1.0 / n) * kf
    kz = np.fft.rfftfreq(n, 1.0 / n) * kf
    kk = np.sqrt(kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2)
    edges = np.linspace(kf, kf * n / 2, n_bins + 1)
    idx = np.digitize(kk.ravel(), edges) - 1
    ok = (idx >= 0) & (idx < n_bins)
    pab = np.bincount(idx[ok], (fa * np.conj(fb)).real.ravel()[ok], n_bins)
    paa = np.bincount(idx[ok], (np.abs(fa) ** 2).ravel()[ok], n_bins)
    pbb = np.bincount(idx[ok], (np.abs(fb) ** 2).ravel()[ok], n_bins)
    return 0.5 * (edges[1:] + edges[:-1]), pab / np.sqrt(paa * pbb)


def _main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description="masked reconstruction, FP32 path vs all-FP64 path")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--box", type=float, default=500.0)
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--precision", choices=["f32", "f64", "both"], default="both")
    ap.add_argument("--steps", type=int, default=10, help="leapfrog steps (the paper's run: 18, da = 0.05)")
    ap.add_argument("--anneal", type=int, default=0,
                    help="coarsening factor of a first, low-resolution stage (0: none; the paper: 4 cMpc/h cells)")
    ap.add_argument("--coarse-iters", type=int, default=250)
    args = ap.parse_args()
    from . import build
    build.build()
    lnk, lnp = api.pm_linear_power_table()
    R, s_true, counts, nbar_cell = masked_mock(args.n, args.box, n_steps=args.steps, lnk=lnk, lnp=lnp)
    s0 = inputs.white_noise(args.n, 2)
    out = {"workload": f"masked-recon-{args.n}", "n": args.n, "box": args.box, "iters": args.iters,
           "steps": args.steps, "galaxies": float(counts.sum()), "nbar_cell": nbar_cell}
    if args.anneal:
        out["workload"] = f"annealed-masked-recon-{args.n // args.anneal}-{args.n}"
        out["coarse_iters"] = args.coarse_iters
    precs = ["f32", "f64"] if args.precision == "both" else [args.precision]
    for prec in precs:
        dt = torch.float32 if prec == "f32" else torch.float64
        dev = lambda x: torch.as_tensor(np.asarray(x)).to(device="cuda", dtype=dt)
        cfg = mock_config(args.n, args.box, nbar_cell, prec, n_steps=args.steps)
        Rd, cd = dev(R), dev(counts)

        def targets_for(plan, Rm):
            nreal = api.pm_count_positive(plan, Rm)
            fcounts = api.pm_rom_fourier_counts(plan)
            return lambda it: (dev(inputs.sorted_normal_targets(nreal, 7 + it)),
                               dev(inputs.sorted_normal_targets_per_bin(fcounts, 7 + it)))

        trace = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if args.anneal:
            nc = args.n // args.anneal
            s, f, info = anneal(cfg, lnk, lnp, dev(inputs.white_noise(nc, 2)), cd, Rd, args.anneal,
                                args.coarse_iters, args.iters, dev(inputs.white_noise(args.n, 8)),
                                targets_for=targets_for, trace=trace)
        else:
            plan = api.Plan(cfg, lnk, lnp)
            s, f, info = reconstruct(plan, dev(s0), cd, Rd, args.iters, rom_targets=targets_for(plan, Rd),
                                     trace=trace)
            plan.close()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        k, r = cross_correlation(s.double().cpu().numpy(), s_true, args.box)
        out[prec] = {"final_loss": f, "seconds": wall, "iters_per_s": args.iters / wall, **info,
                     "loss_trace": [(i, l) for i, l in trace if i % max(1, args.iters // 10) == 0],
                     "r_k": {"k": [round(x, 4) for x in k[:8]], "r": [round(x, 4) for x in r[:8]]}}
        del s
        torch.cuda.empty_cache()
    if "f32" in out and "f64" in out:
        out["final_loss_rel_diff"] = abs(out["f32"]["final_loss"] - out["f64"]["final_loss"]) / abs(
            out["f64"]["final_loss"])
        out["speedup_f32_over_f64"] = out["f64"]["seconds"] / out["f32"]["seconds"]
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    _main()
