"""Per-stage agreement of the FP32 path with the all-FP64 path on the masked
256^3 workload (the FP64 GPU path agrees with the FP64 oracle to ~1e-11 at
the sizes the oracle can run, so it stands in for the oracle at 256^3).

Stages, each evaluated by both precisions from the same white noise s0:
linear field delta_L, 2LPT displacement and momentum, the force at the 2LPT
state, the displacement and momentum after the 10 leapfrog steps, the force
at that final state, the final density contrast, the loss, and the gradient
(relative L2 and cosine).  Prints one JSON line.
"""
import json

import numpy as np
import torch

from . import api, build, inputs, recon


def rel_l2(a, b):
    a = a.double().reshape(-1)
    b = b.double().reshape(-1)
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def cosine(a, b):
    a = a.double().reshape(-1)
    b = b.double().reshape(-1)
    return float(torch.dot(a, b) / (torch.linalg.norm(a) * torch.linalg.norm(b)))


def main(n=256, box=500.0):
    build.build()
    lnk, lnp = api.pm_linear_power_table()
    R, s_true, counts, nbar_cell = recon.masked_mock(n, box, lnk=lnk, lnp=lnp)
    s0 = inputs.white_noise(n, 2)
    res = {}
    for prec in ("f64", "f32"):
        dt = torch.float32 if prec == "f32" else torch.float64
        dev = lambda x: torch.as_tensor(np.asarray(x)).to(device="cuda", dtype=dt)
        plan = api.Plan(recon.mock_config(n, box, nbar_cell, prec), lnk, lnp)
        s, c, r = dev(s0), dev(counts), dev(R)
        out = {"delta_L": api.pm_linear_field(plan, s)}
        out["lpt_disp"], out["lpt_mom"] = api.pm_lpt(plan, s)
        out["force_lpt"] = api.pm_force(plan, out["lpt_disp"])
        out["final_disp"], out["final_mom"] = api.pm_evolve(plan, s)
        out["force_final"] = api.pm_force(plan, out["final_disp"])
        delta = plan.empty()
        out["loss"] = api.pm_forward(plan, s, c, r, delta_out=delta)
        out["delta_final"] = delta
        _, out["grad"] = api.pm_adjoint(plan, s, c, r)
        res[prec] = {k: (v.double().cpu() if torch.is_tensor(v) else v) for k, v in out.items()}
        plan.close()
        del plan, out, delta
        torch.cuda.empty_cache()
    a, b = res["f32"], res["f64"]
    stages = {k: rel_l2(a[k], b[k]) for k in a if k != "loss"}
    line = {"workload": f"masked-recon-{n}", "reference": "all-FP64 GPU path", "rel_l2_fp32_vs_fp64": stages,
            "loss_rel_diff": abs(a["loss"] - b["loss"]) / abs(b["loss"]),
            "grad_cosine": cosine(a["grad"], b["grad"])}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
