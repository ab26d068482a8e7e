"""Timings of the paper's full run recipe on one GPU (Sec. 2.2.1, Sec. 3,
Appendix A), beyond the benchmark workload:

  lightcone   gradient evaluations per second at n^3 (default 256^3 in
              500 Mpc/h) with 18 leapfrog steps (da = 0.05 from a = 0.1),
              snapshots at a = 0.8, 0.9, 1, the lightcone and the radial
              redshift-space shift seen from (250, 250, -150) Mpc/h, masked
              Poisson likelihood;
  coarse      the same at (n/2)^3, the annealing stage's mesh;
  analysis    P(k) auto + cross spectra (32 bins) and the T-web
              (R_sm = 2 Mpc/h, lambda_th = 0.16) of two n^3 fields;
  fma_tflops  the measured FP32 / FP64 FMA rates (the arithmetic ceiling
              against which the all-FP64 path is read).

Every number is CUDA-event time on the launching (default) stream after
warm-up; inputs are resident on the device.  One JSON line:

    python -m paper_2604_26823_gb300.recipe --n 256 --evals 5
"""
import argparse
import json

import torch

from . import api, build, inputs, recon

OBSERVER = (250.0, 250.0, -150.0)


def _timed(fn, reps, warm=2):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        fn()
    t1.record()
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / reps   # ms per call


def lightcone_rate(n, box, steps, evals, lnk, lnp):
    """(gradient evaluations per second, loss) of the lightcone model at n^3."""
    R, _, counts, nbar = recon.masked_mock(n, box, n_steps=steps, lnk=lnk, lnp=lnp)
    cfg = recon.mock_config(n, box, nbar, n_steps=steps)
    cfg.rsd_axis, cfg.lightcone, cfg.observer = 3, True, OBSERVER
    plan = api.Plan(cfg, lnk, lnp)
    dev = lambda x: torch.tensor(x, dtype=torch.float32, device="cuda")
    s, c, r = dev(inputs.white_noise(n, 2)), dev(counts), dev(R)
    g = torch.empty_like(s)
    out = {}

    def step():
        out["loss"], _ = api.pm_adjoint(plan, s, c, r, grad_out=g)

    ms = _timed(step, evals)
    plan.close()
    return 1e3 / ms, out["loss"]


def analysis_times(n, box, reps, lnk, lnp):
    """(ms of pm_power_spectra on two fields, ms of pm_tweb with eigenvectors)."""
    plan = api.Plan(api.Config(n=n, box=box, n_steps=2), lnk, lnp)
    dev = lambda x: torch.tensor(x, dtype=torch.float32, device="cuda")
    a = dev(inputs.normal_field(n, 41))
    b = dev(inputs.normal_field(n, 42))
    ms_pk = _timed(lambda: api.pm_power_spectra(plan, a, b, 32), reps)
    ms_tw = _timed(lambda: api.pm_tweb(plan, a, 2.0, 0.16), reps)
    plan.close()
    return ms_pk, ms_tw


def main():
    ap = argparse.ArgumentParser(description="timings of the paper's run recipe")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--box", type=float, default=500.0)
    ap.add_argument("--steps", type=int, default=18)
    ap.add_argument("--evals", type=int, default=5)
    args = ap.parse_args()
    build.build()
    lnk, lnp = api.pm_linear_power_table()
    res = {"workload": f"recipe-{args.n}", "n": args.n, "box": args.box, "steps": args.steps, "dtype": "f32",
           "observer": OBSERVER}
    rate, loss = lightcone_rate(args.n, args.box, args.steps, args.evals, lnk, lnp)
    res["lightcone"] = {"evals_per_s": rate, "loss": loss}
    torch.cuda.empty_cache()
    rate_c, loss_c = lightcone_rate(args.n // 2, args.box, args.steps, 2 * args.evals, lnk, lnp)
    res["coarse"] = {"n": args.n // 2, "evals_per_s": rate_c, "loss": loss_c}
    torch.cuda.empty_cache()
    ms_pk, ms_tw = analysis_times(args.n, args.box, args.evals, lnk, lnp)
    res["analysis"] = {"power_spectra_ms": ms_pk, "tweb_ms": ms_tw}
    res["fma_tflops"] = {"f32": api.pm_fma_rate("f32", 16384), "f64": api.pm_fma_rate("f64", 4096)}
    res["peak_allocated_gb"] = torch.cuda.max_memory_allocated() / 1e9
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
