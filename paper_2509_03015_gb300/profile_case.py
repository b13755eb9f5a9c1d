"""Run one named workload through the library a fixed number of times, for
profiling (ncu launch lists and captures).

  python -m paper_2509_03015_gb300.profile_case --workload kalman-N4096-n256-d16-rho0.99 \
      --precision fp32_ir [--per-level] [--reps 1] [--N 512]
"""
from __future__ import annotations

import argparse
import time

import torch

from . import Solver, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="kalman-N16384-n64-d4", choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_ir", "tf32_ir"])
    ap.add_argument("--per-level", action="store_true")
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--N", type=int, default=None, help="horizon override (same generator)")
    args = ap.parse_args()
    cfg = dict(inputs.WORKLOADS[args.workload])
    if args.N is not None:
        cfg["N"] = args.N
    s = inputs.kalman_btd(cfg["N"], cfg["n"], cfg["m"], cfg["d"], cfg["rho"], cfg["seed"])
    dev = torch.device("cuda:0")
    Ad, As, B = (torch.from_numpy(s[k]).to(dev) for k in ("A_diag", "A_sub", "B"))
    sol = Solver(cfg["N"], cfg["n"], d_max=cfg["d"], precision=args.precision, persistent=not args.per_level)
    X = torch.empty_like(B)
    for _ in range(args.reps):
        t0 = time.perf_counter()
        sol.factor_solve(Ad, As, B, X)
        torch.cuda.synchronize()
        info = sol.last_info
        print(f"{args.workload} N={cfg['N']} {args.precision} per_level={args.per_level}: "
              f"{1e3 * (time.perf_counter() - t0):.2f} ms, iters {info.iters}, berr {info.backward_err:.2e}, "
              f"launches {sol.launch_stats()[0]}")
    sol.close()


if __name__ == "__main__":
    main()
