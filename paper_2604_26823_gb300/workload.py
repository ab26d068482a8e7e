"""A fixed workload for profilers: ``evals`` gradient evaluations (pm_adjoint)
of the masked Poisson reconstruction problem at n^3 (box scaled with n so
the cell stays 500/256 Mpc/h), FP32 path, after the mock and the plan are
built.  Nothing is timed here; run it under ncu, e.g.

    python -m paper_2604_26823_gb300.workload --n 256 --evals 2
"""
import argparse

import torch

from . import api, build, inputs, recon


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--evals", type=int, default=2)
    ap.add_argument("--steps", type=int, default=10, help="leapfrog steps")
    args = ap.parse_args()
    build.build()
    n, box = args.n, 500.0 * args.n / 256
    lnk, lnp = api.pm_linear_power_table()
    R, _, counts, nbar = recon.masked_mock(n, box, n_steps=args.steps, lnk=lnk, lnp=lnp)
    plan = api.Plan(recon.mock_config(n, box, nbar, n_steps=args.steps), lnk, lnp)
    dev = lambda x: torch.tensor(x, dtype=torch.float32, device="cuda")
    s0, c, r = dev(inputs.white_noise(n, 2)), dev(counts), dev(R)
    loss = None
    for _ in range(args.evals):
        loss, _ = api.pm_adjoint(plan, s0, c, r)
    torch.cuda.synchronize()
    print(f"n={n} evals={args.evals} loss={loss:.6f} peak_allocated_gb={torch.cuda.max_memory_allocated() / 1e9:.2f}")


if __name__ == "__main__":
    main()
