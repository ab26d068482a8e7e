#!/usr/bin/env python
"""Gradient evaluations per second of the MujicΛ hot path on one GB300.

Workload: the masked-reconstruction configuration -- 256^3 mesh and
particles, 500 Mpc/h box, 2LPT to a = 0.1 then 10 leapfrog steps to a = 1,
power-law + sigmoid bias (0.7, 1.2, 3.0) with a survey response R (40 deg
cone, radial n(r) ~ r^2 exp(-(r/300)^1.5), 16x16 angular completeness
patches U(0.3, 0.9)), Poisson likelihood on mock counts drawn at
nbar = 1e-3 (h/Mpc)^3, Gaussian prior, m = 10 L-BFGS.

One step = one augmented L-BFGS iteration of the hot path: lbfgs_step
(pair push + two-loop direction), the trial point s + eps p_hat (eps =
min(|d|, 1)), project_rank_match (projection every step; Fourier and
real-space rank-order matching on every 20th step, the paper's schedule),
and pm_adjoint (forward model + gradient) at the trial point.  Each step is
exactly one gradient evaluation, so steps/s = gradient evals/s.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PM fwd+adjoint gradient evals/s at 256^3 (FP32 mesh/FFT/particles, FP64 reductions)"
UNIT = "gradient evals/s"
N, BOX, STEPS_PM = 256, 500.0, 10
NBAR = 1e-3
ROM_EVERY = 20
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, mean
# over the cotangent-paint launches of one gradient evaluation of this
# workload, k = 9 .. 0) from one ncu capture of the kernel as it stands;
# profiles/deposit_traffic_masked_recon_256.md gives the command.  Set to None
# when the kernel changes.
NCU_TRAFFIC = {"adj_paint": 1152.3e6}

def config(api, nbar_cell, precision="f32"):
    from paper_2604_26823_gb300 import recon
    return recon.mock_config(N, BOX, nbar_cell, precision, n_steps=STEPS_PM)


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(backend=None):
    """Rank / world size from the launcher's environment; with several ranks,
    a process group (NCCL on GPUs; gloo when given or without CUDA)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return ws, rank, local


def replica_seeds(rank):
    """Seeds of one replica: each rank reconstructs its own mock (replicas
    only; no data-path collective)."""
    return {"truth": 1 + 1000 * rank, "counts": 3 + 1000 * rank, "start": 2 + 1000 * rank}


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ws, seconds_local):
    """Units all ranks processed / the slowest rank's time (max over ranks)."""
    return ws * units_per_rank / max_over_ranks(seconds_local, ws)


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_sample(n_small=64):
    """One FP64 oracle gradient of the same physics at n_small^3 (same cell
    size), seconds; scaled to 256^3 by the cell count."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import cosmology as OC
    from oracle import model as OM
    from paper_2604_26823_gb300 import inputs
    box = BOX * n_small / N
    lnk, lnp = OC.linear_power_table()
    cfg = OM.Config(n=n_small, box=box, n_steps=STEPS_PM, lpt_order=2, likelihood="poisson",
                    nbar_cell=NBAR * (BOX / N) ** 3, alpha=0.7, delta_th=1.2, K=3.0, prior_weight=1.0)
    s = inputs.white_noise(n_small, 2).astype(np.float64)
    resp = inputs.survey_selection(n_small, box, 4, observer=(box / 2, box / 2, -0.3 * box),
                                   r_scale=300.0 * n_small / N).astype(np.float64)
    counts = inputs.poisson_counts(resp * NBAR * (BOX / N) ** 3, 3).astype(np.float64)
    OC.growth([0.1], 0.25)  # warm the growth cache outside the timing
    t0 = time.perf_counter()
    OM.gradient(s, cfg, lnk, lnp, counts, resp)
    return time.perf_counter() - t0, (N / n_small) ** 3


def run_reference(args, ws, rank):
    if rank != 0:
        return
    n_small = 32
    for _ in range(args.warmup):
        oracle_sample(n_small)
    times = []
    for _ in range(args.steps):
        t, scale = oracle_sample(n_small)
        times.append(t * scale)
    per = float(np.mean(times))
    value = 1.0 / per
    sample = (f"one FP64 oracle gradient (2LPT + 10 steps, Poisson, same cell size) at {n_small}^3 per step, "
              f"time scaled x{int((N / n_small) ** 3)} by cell count to 256^3")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "masked-recon-256", "n_mesh": N, "n_particles": N ** 3, "box": BOX,
                       "pm_steps": STEPS_PM, "parallelism": f"replicas x{args.gpus}"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fft_comparison(api, plan, s, reps=20):
    import torch
    out = torch.empty_like(s)
    amp = torch.rand((N, N, N // 2 + 1), dtype=torch.float32, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(f):
        for _ in range(3):
            f()
        a, b = ev(), ev()
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            f()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    ours = timed(lambda: api.pm_linear_field(plan, s, out=out))
    cufft = timed(lambda: torch.fft.irfftn(torch.fft.rfftn(s) * amp, s=(N, N, N)))
    return {"op": "linear field: real 256^3 -> spectrum x A(k) -> real (FP32)", "library_ms": ours,
            "cufft_ms": cufft, "note": "comparison only; cuFFT is not used on the path"}


def run_ckpt512(api, inputs, lnk, lnp, evals=3):
    """pm_adjoint at 512^3 in a 1000 Mpc/h box, 2LPT + 10 steps, Gaussian
    likelihood with b = 1.5 over the full box, particle states checkpointed
    every 2 steps; data is a seeded N(0,1) field (the cost does not depend on
    its values)."""
    import torch
    n = 512
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    free0, total = torch.cuda.mem_get_info()
    cfg = api.Config(n=n, box=1000.0, n_steps=STEPS_PM, lpt_order=2, rsd_axis=-1, likelihood="gaussian",
                     bias_b=1.5, sigma=1.0, prior_weight=1.0, checkpoint_every=2)
    plan = api.Plan(cfg, lnk, lnp)
    s = torch.from_numpy(inputs.white_noise(n, 1)).cuda()
    d = torch.from_numpy(inputs.normal_field(n, 3)).cuda()
    R = torch.ones((n, n, n), dtype=torch.float32, device="cuda")
    g = torch.empty_like(s)
    api.pm_adjoint(plan, s, d, R, grad_out=g)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(evals):
        api.pm_adjoint(plan, s, d, R, grad_out=g)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / evals
    free1, _ = torch.cuda.mem_get_info()
    out = {"workload": "ckpt-512", "n_mesh": n, "box": 1000.0, "pm_steps": STEPS_PM, "checkpoint_every": 2,
           "value": 1e3 / ms, "unit": UNIT, "ms_per_eval": ms, "evals": evals,
           "workspace_gb": plan.workspace_bytes / 1e9,
           "peak_torch_allocated_gb": torch.cuda.max_memory_allocated() / 1e9,
           "device_used_gb": (total - free1) / 1e9}
    plan.close()
    del plan, s, d, R, g
    torch.cuda.empty_cache()
    return out


def run_ours(args, ws, rank, local):
    import torch
    from paper_2604_26823_gb300 import api, build, inputs, recon
    build.build()
    lib = api.L.load()
    torch.cuda.set_device(local)
    lnk, lnp = api.pm_linear_power_table()
    dev = lambda x: torch.tensor(x, dtype=torch.float32, device="cuda")

    seeds = replica_seeds(rank)
    R_h, s_true, counts_h, nbar_cell = recon.masked_mock(N, BOX, n_steps=STEPS_PM, nbar=NBAR,
                                                         seed_truth=seeds["truth"], seed_counts=seeds["counts"],
                                                         lnk=lnk, lnp=lnp)
    cfg = config(api, nbar_cell)
    plan = api.Plan(cfg, lnk, lnp)
    R = dev(R_h)
    counts = dev(counts_h)
    n_gal = float(counts_h.sum())
    vol_frac = float((R_h > 0).mean())
    ncount = api.pm_count_positive(plan, R)
    t_real = dev(inputs.sorted_normal_targets(ncount, 7))
    t_four = dev(inputs.sorted_normal_targets_per_bin(api.pm_rom_fourier_counts(plan), 8))
    st = api.LBFGS(N ** 3, m=10, precision="f32")
    s0 = inputs.white_noise(N, seeds["start"])
    state = {"s": dev(s0), "g": torch.empty((N, N, N), dtype=torch.float32, device="cuda"),
             "trial": torch.empty((N, N, N), dtype=torch.float32, device="cuda"), "it": 0}
    _, state["g"] = api.pm_adjoint(plan, state["s"], counts, R, grad_out=state["g"])

    def step(plan_, st_, S, cnt, resp, tr, tf):
        it = S["it"]
        d, gd, dn, _ = api.lbfgs_step(st_, S["s"], S["g"])
        eps = min(dn, 1.0)
        api.pm_axpy(eps / dn, d, S["s"], out=S["trial"])
        mode = api.L.PM_PROJECT | (api.L.PM_ROM_FOURIER | api.L.PM_ROM_REAL if it % ROM_EVERY == 0 else 0)
        api.project_rank_match(plan_, S["trial"], mode, R=resp, targets_real=tr, targets_fourier=tf, seed=6,
                               counter=it)
        loss, _ = api.pm_adjoint(plan_, S["trial"], cnt, resp, grad_out=S["g"])
        S["s"], S["trial"] = S["trial"], S["s"]
        S["it"] = it + 1
        return loss

    for _ in range(args.warmup):
        step(plan, st, state, counts, R, t_real, t_four)
    state["it"] = 0
    torch.cuda.synchronize()
    barrier(ws)
    clocks = Clocks(local)
    api.pm_profile(plan, True, 200000)
    launches0 = lib.pm_launch_count()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    losses = []
    torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select exactly the timed launches
    for _ in range(args.steps):
        losses.append(step(plan, st, state, counts, R, t_real, t_four))
    torch.cuda.nvtx.range_pop()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = lib.pm_launch_count() - launches0
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    prof = {c: api.pm_profile_read(plan, c) for c in api.PROFILE_CLASSES}
    api.pm_profile(plan, False)
    barrier(ws)
    value = whole_job_rate(args.steps, ws, ms / 1e3)
    ms_max = ws * args.steps / value * 1e3

    # dominant kernel class: algorithmic bytes (recorded per launch by the
    # library) over its event-timed duration, against the measured HBM peak
    peak, peak_src = 6800.0, "fallback (6.8 TB/s)"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak, peak_src = float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        pass
    classes = {k: {"ms_total": v[0], "launches": v[1], "GBps": (v[2] / (v[0] / 1e3) / 1e9) if v[0] else None}
               for k, v in prof.items()}
    # byte model of the step: the algorithmic bytes the library records for its
    # profiled kernel classes (inputs read once, outputs written once), per
    # step, over the measured step time (end-to-end effective bandwidth)
    alg_step = sum(v[2] for v in prof.values()) / args.steps
    bytes_model = {"algorithmic_bytes_per_step": alg_step, "profiled_classes_ms_per_step":
                   sum(v[0] for v in prof.values()) / args.steps,
                   "effective_GBps": alg_step / (ms / args.steps / 1e3) / 1e9}
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_n, dom_b = prof[dom]
    roof = None
    if dom_n:
        achieved = dom_b / (dom_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": NCU_TRAFFIC.get(dom), "peak_source": peak_src, "launches": dom_n,
                "mean_launch_ms": dom_ms / dom_n, "algorithmic_bytes_per_launch": dom_b / dom_n,
                "share_of_step": dom_ms / ms}
    # FP64 path: same workload and schedule
    fp64 = None
    if not args.no_fp64:
        del plan
        torch.cuda.empty_cache()
        plan64 = api.Plan(config(api, nbar_cell, "f64"), lnk, lnp)
        d64 = lambda x: torch.as_tensor(x).to(device="cuda", dtype=torch.float64)
        st64 = api.LBFGS(N ** 3, m=10, precision="f64")
        S64 = {"s": d64(s0), "g": torch.empty((N, N, N), dtype=torch.float64, device="cuda"),
               "trial": torch.empty((N, N, N), dtype=torch.float64, device="cuda"), "it": 0}
        c64, R64 = d64(counts_h), d64(R_h)
        tr64, tf64 = d64(t_real.cpu().numpy()), d64(t_four.cpu().numpy())
        _, S64["g"] = api.pm_adjoint(plan64, S64["s"], c64, R64, grad_out=S64["g"])
        step(plan64, st64, S64, c64, R64, tr64, tf64)
        S64["it"] = 0
        torch.cuda.synchronize()
        k64 = max(2, min(args.steps, 4))
        t0 = time.perf_counter()
        for _ in range(k64):
            step(plan64, st64, S64, c64, R64, tr64, tf64)
        torch.cuda.synchronize()
        fp64 = {"value": k64 / (time.perf_counter() - t0), "unit": UNIT, "steps": k64}
        del plan64, st64, S64
        torch.cuda.empty_cache()
        plan = api.Plan(cfg, lnk, lnp)

    # checkpointed 512^3 configuration (1000 Mpc/h, 10 steps, states kept every
    # 2 steps): gradient evals/s and peak device memory
    # cuFFT as a comparison only: the linear field delta_L = IFFT[A(k) FFT[s]]
    # through the library's pencil passes (one r2c, y, fused x with the
    # amplitude multiplier, y, c2r) against torch.fft (cuFFT) rfftn * A irfftn
    # on the same 256^3 FP32 mesh (the cuFFT side skips the DC / Nyquist
    # conventions, so only the times are compared)
    fft_cmp = fft_comparison(api, plan, state["s"])

    ck512 = None
    if not args.no_512:
        del plan
        torch.cuda.empty_cache()
        ck512 = run_ckpt512(api, inputs, lnk, lnp)
        plan = api.Plan(cfg, lnk, lnp)

    # end to end through the public API with pinned host buffers: every step
    # uploads s, the counts and R and reads back the loss
    s_pin = torch.from_numpy(state["s"].cpu().numpy()).pin_memory()
    c_pin = torch.from_numpy(counts_h).pin_memory()
    r_pin = torch.from_numpy(R_h).pin_memory()
    S2 = {"s": torch.empty_like(state["s"]), "g": torch.empty_like(state["g"]),
          "trial": torch.empty_like(state["s"]), "it": 1}
    cnt2, R2 = torch.empty_like(counts), torch.empty_like(R)
    st2 = api.LBFGS(N ** 3, m=10, precision="f32")
    S2["s"].copy_(s_pin, non_blocking=True)
    cnt2.copy_(c_pin, non_blocking=True)
    R2.copy_(r_pin, non_blocking=True)
    _, S2["g"] = api.pm_adjoint(plan, S2["s"], cnt2, R2, grad_out=S2["g"])
    torch.cuda.synchronize()
    k_e2e = args.steps
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        S2["s"].copy_(s_pin, non_blocking=True)
        cnt2.copy_(c_pin, non_blocking=True)
        R2.copy_(r_pin, non_blocking=True)
        step(plan, st2, S2, cnt2, R2, t_real, t_four)   # returns the loss on the host
    torch.cuda.synchronize()
    e2e_t = time.perf_counter() - t0
    e2e_t = max_over_ranks(e2e_t, ws)
    e2e = {"value": ws * k_e2e / e2e_t, "unit": UNIT, "h2d_bytes_per_step": 3 * 4 * N ** 3,
           "d2h_bytes_per_step": 8}

    cpu = None
    if rank == 0 and not args.no_cpu:
        t, scale = oracle_sample(64)
        cpu = {"value": 1.0 / (t * scale), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one FP64 oracle gradient (same physics and cell size) at 64^3 took {t:.1f} s, "
                         f"scaled x{int(scale)} by cell count to 256^3"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "masked-recon-256", "n_mesh": N, "n_particles": N ** 3, "box": BOX,
                           "pm_steps": STEPS_PM, "lbfgs_m": 10, "rom_every": ROM_EVERY,
                           "likelihood": "poisson", "galaxies": n_gal, "selection_volume_frac": vol_frac,
                           "parallelism": f"replicas x{ws}", "l2": "working set ~7 GB >> 129 MB L2 (no flush)"},
                "fp64_path": fp64, "checkpointed_512": ck512, "fft_vs_cufft": fft_cmp, "e2e": e2e, "roofline": roof, "cpu_baseline": cpu,
                "gpu_launches": int(launches), "clocks": clk, "kernel_classes": classes, "bytes_model": bytes_model,
                "final_loss": losses[-1]}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-512", action="store_true", help="skip the checkpointed 512^3 measurement")
    args = ap.parse_args()
    ws, rank, local = (1, 0, 0) if args.impl == "reference" and int(os.environ.get("WORLD_SIZE", "1")) == 1 \
        else dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
