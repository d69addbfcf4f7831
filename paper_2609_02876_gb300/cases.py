"""Run one named workload once, for profiling a single kernel under ncu.

    python -m paper_2609_02876_gb300.cases <case> [--traj N] [--problem P] [--precision fp64|fp32_mixed]
                                                  [--method tsit5|rodas5p|rosenbrock23|verner7]

Cases (each on the seeded synthetic workload of `workloads.make`):
  solve_grad    record + reverse sweep (gs_solve_grad), 3 warm-up calls then one
  forward_only  gs_solve (nothing recorded), 3 warm-up calls then one
  jvp           record once, then forward-mode gradient w.r.t. theta (gs_forward_grad),
                3 warm-up calls then one
The last call of each case is the one to capture (ncu -s / -c by kernel name).
"""
from __future__ import annotations

import argparse
import sys

import numpy as np
import torch

from . import api, build
from . import workloads as W


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["solve_grad", "forward_only", "jvp"])
    ap.add_argument("--traj", type=int, default=1 << 20)
    ap.add_argument("--problem", default="lorenz")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_mixed"])
    ap.add_argument("--method", default=None, choices=["tsit5", "rodas5p", "rosenbrock23", "verner7"],
                    help="default: Tsit5 for the non-stiff problems, Rodas5P for the stiff ones")
    args = ap.parse_args(argv)
    build.build()
    wl = W.make(args.problem, args.traj)
    P = torch.as_tensor(np.ascontiguousarray(wl["params"].T), device="cuda")
    Y = torch.as_tensor(np.ascontiguousarray(wl["y0"].T), device="cuda")
    SW = None if wl["w"] is None else torch.as_tensor(np.asarray(wl["w"], dtype=np.float32), device="cuda")
    common = (wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"])
    if args.case == "solve_grad":
        run = lambda: api.solve_grad(args.problem, P, Y, *common, layout="soa", precision=args.precision,
                                     shared_w=SW, method=args.method)
    elif args.case == "forward_only":
        run = lambda: api.solve(args.problem, P, Y, *common, layout="soa", precision=args.precision, shared_w=SW,
                                method=args.method)
    else:
        rec, _, _ = api.forward_record(args.problem, P, Y, *common, layout="soa", want_saves=False,
                                       method=args.method)
        run = lambda: api.forward_grad(rec, P, Y, wrt=("params",), layout="soa")
    for _ in range(4):
        run()
    torch.cuda.synchronize()
    print(f"{args.case} {args.problem} n={args.traj} {args.precision}: ok", flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
