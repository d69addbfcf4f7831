#!/usr/bin/env python3
"""Benchmark: gradient trajectories/s of the record + reverse-sweep hot path.

One step = one gs_solve_grad call over a resident ensemble: the adaptive Tsit5
record of every trajectory, then the reverse discrete-adjoint sweep with the
built-in loss sum_s ||y(t_s)||^2, returning loss, dL/dtheta and dL/dy0.

Default workload (the non-stiff scale sweep's largest Lorenz point): Lorenz-63,
n = 2^24 trajectories per GPU, sigma~U[8,12], rho~U[20,30], beta~U[2,3],
y0~N((1,1,1), 0.1^2 I), t in [0, 1], 10 uniform save times, Tsit5 with
rtol 1e-6 / atol 1e-8, FP64. Inputs (805 MB) and the record (~10 GB) are far
larger than L2, so no flush is needed between steps.

Launch: python bench.py [--gpus N --steps K --warmup W] on one GPU, or under
torchrun (one rank per GPU, each rank its own shard: weak scaling).
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2609_02876_gb300 import workloads as W  # noqa: E402

METRIC = "gradient trajectories/s on 1 GB300 at matched error vs FP64 oracle; p50/p99 latency"
UNIT = "trajectories/s"

# Hand-counted algorithmic flops (FMA = 2) per unit, from the operations each step performs.
# Per problem: f = one right-hand side, vjp = one J^T v + f_theta^T v,
# jac = the dense Jacobian, con = one gradient of r^T J u (stiff problems), D.
RHS_FLOPS = {"lorenz": dict(f=8, vjp=20, D=3), "vdp": dict(f=5, vjp=15, D=2),
             "robertson": dict(f=8, vjp=19, jac=5, con=23, D=3),
             "hires": dict(f=36, vjp=80, jac=4, con=49, D=8),
             # LV UDE: MLP 2-16-16-2 forward (W1 64, W2 512, W3 64 flops, 32 tanh at ~5) plus the
             # linear terms; the VJP recomputes the forward and back-propagates (~750 more); the
             # shared-weight gradient contraction runs on the tensor cores and is not counted here
             "lv_ude": dict(f=804, vjp=1554, D=2),
             # neural Robertson (FP64 MLP 3-16-16-1): f = 320 FMAs + the Robertson terms (tanh,
             # exp, log1p counted as one flop each); the VJP adds the backward pass and the
             # warp's weight contraction (353 weights x 32 lanes x 2 / 32 lanes); J is one
             # forward + backward pass; the contraction a tangent pass, a double backward pass
             # and two weight contractions
             "nrob": dict(f=690, vjp=2050, jac=1330, con=4100, D=3)}
STIFF = {"robertson", "hires", "nrob"}


# DRAM bytes per accepted step, read + write, measured with ncu (dram__bytes_read.sum +
# dram__bytes_write.sum, one launch of each kernel) on the first 2^20 trajectories of
# the same FP64 workload (Lorenz: 45.15 accepted steps per trajectory; Robertson:
# 101243901 accepted steps in all), per record layout; a launch's traffic grows in
# proportion to its accepted steps.
TRAFFIC_PER_STEP = {("lorenz", "fp64", "reverse", "compact"): (4625075712 + 71750656) / (45.15 * 2 ** 20),
                    ("lorenz", "fp64", "record", "compact"): (66017280 + 2269651712) / (45.15 * 2 ** 20),
                    ("lorenz", "fp64", "reverse", "stages"): (15005185536 + 89034752) / (45.15 * 2 ** 20),
                    ("lorenz", "fp64", "record", "stages"): (1782274816 + 11522356736) / (45.15 * 2 ** 20),
                    ("robertson", "fp64", "reverse", "stages"): (49914448640 + 67795200) / 101243901,
                    ("robertson", "fp64", "record", "stages"): (3282266112 + 66818809344) / 101243901}


def unit_flops(problem, method=None):
    c = RHS_FLOPS[problem]
    f, v, D = c["f"], c["vjp"], c["D"]
    norm = 6 * D + 4  # weighted RMS error test and step control
    if method == "rosenbrock23":
        # W = I - h d J (J, D^2 scale, D), LU (2/3 D^3); k1 and u2 solves (2 D^2 each),
        # Y1 (2 D), f(Y1), F1 - k1 (D), y_new (3 D): the replay step with f(y).
        # Trial adds f(y_new), the k3 right-hand side (6 D), its solve and e (5 D).
        # Reverse: two transposed solves, two VJPs, 8 D of recursions, two contractions.
        step = c["jac"] + D * D + D + (2 * D ** 3) // 3 + 4 * D * D + 6 * D + 2 * f
        trial = step + 2 * D * D + 11 * D + norm  # f(y) carried from the last step, f(y_new) added
        rev = 4 * D * D + 2 * v + 8 * D + 2 * c["con"]
        return {"stage_fwd": step, "vjp_unit": step + rev, "trial": trial}
    if method == "verner7":
        # Verner7 (10 stages, 36 nonzero a_ij, 30 of them in stages 2..9): the replay
        # step evaluates 9 slopes, the stage inputs (sum over rows of 2 m + 1 per
        # component for m coefficients: 68 D) and y_new (7 weights: 15 D). The trial
        # adds stage 10 (f, 13 D) and the error estimate (8 weights: 16 D). Reverse:
        # 9 stage VJPs, the a_ij recursions (60 D), kbar and the cotangent sum (34 D).
        step = 9 * f + 83 * D
        trial = 10 * f + 112 * D + norm
        rev = 9 * v + 94 * D
        return {"stage_fwd": step, "vjp_unit": step + rev, "trial": trial}
    if problem not in STIFF:
        # Tsit5: stage forward (6 slopes + 6 stage inputs) 6 f + 48 D;
        # stage reverse (6 stage VJPs + cotangent recursion) 6 vjp + 54 D
        fwd = 6 * f + 48 * D
        rev = 6 * v + 54 * D
        trial = 7 * f + 48 * D + 14 * D + norm
        return {"stage_fwd": fwd, "vjp_unit": fwd + rev, "trial": trial}
    # Rodas5P (8 stages): J, W = I/(h gamma) - J, LU (2/3 D^3), per stage the
    # stage input (2 i D), f, the right-hand side (2 i D + 2 D) and one solve
    # (2 D^2); y_new (D). Reverse: per stage one transposed solve (2 D^2), the
    # C and a recursions (4 i D + D), one VJP, one Jacobian contraction.
    step = c["jac"] + D + (2 * D ** 3) // 3 + 56 * D + 8 * f + 70 * D + 16 * D * D + D
    rev = 7 * D + 16 * D * D + 8 * D + 112 * D + 8 * v + 8 * D + 8 * c["con"]
    return {"stage_fwd": step, "vjp_unit": step + rev, "trial": step + D + norm}


def fp_peak_tflops(precision):
    """ALU peak from unit counts and clock: 152 SMs x FMA lanes/clk/SM x 2 x 2.07 GHz.
    FP64 lanes/clk/SM were measured on this part with a dependent-FMA probe."""
    lanes = {"fp64": FP64_LANES_PER_SM, "fp32_mixed": 128}[precision]
    return 152 * lanes * 2 * 2.070e9 / 1e12


FP64_LANES_PER_SM = 2  # DFMA probe on this part: 1.06 TFLOP/s sustained


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_method(args):
    import oracle
    return {"rosenbrock23": oracle.METHOD_ROSENBROCK23, "verner7": oracle.METHOD_VERNER7}.get(args.method,
                                                                                              oracle.METHOD_AUTO)


def cpu_baseline(args, budget_s=12.0):
    """The FP64 oracle (record + replay gradient), as it stands, on the host cores,
    over a bounded sample of the same workload."""
    import oracle
    cores = os.cpu_count() or 1
    om = oracle_method(args)
    probe = W.make(args.problem, 2048, rtol=args.rtol, seed=7)
    t = time.perf_counter()
    oracle.solve_grad(probe["problem"], probe["params"], probe["y0"], probe["t0"], probe["t1"], probe["save_t"],
                      probe["rtol"], probe["atol"], nthreads=cores, method=om, w=probe["w"])
    rate = 2048 / (time.perf_counter() - t)
    m = int(min(max(4096, rate * budget_s), 1 << 22))
    wl = W.make(args.problem, m, rtol=args.rtol, seed=0)
    t = time.perf_counter()
    g = oracle.solve_grad(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                          wl["atol"], nthreads=cores, method=om, w=wl["w"])
    dt = time.perf_counter() - t
    assert g["ok"].all()
    return {"value": m / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {m} trajectories of the same {args.problem} workload (seed 0), record + replay "
                      f"gradient, {dt:.1f} s on {cores} threads"}


def accuracy_sample(args, precision, m=512):
    """Gradient error against the FP64 oracle on the GPU's own mesh, over the
    first m trajectories of the same workload: normwise relative error of each
    trajectory's (theta_bar, y0_bar) vector, median and max."""
    import torch

    import oracle
    from paper_2609_02876_gb300 import api
    wl = W.make(args.problem, m, rtol=args.rtol, seed=0)
    P = torch.as_tensor(np.ascontiguousarray(wl["params"].T), device="cuda")
    Y = torch.as_tensor(np.ascontiguousarray(wl["y0"].T), device="cuda")
    SW = None if wl["w"] is None else torch.as_tensor(np.asarray(wl["w"], dtype=np.float32), device="cuda")
    rec, _, _ = api.forward_record(args.problem, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                                   layout="soa", want_saves=False, precision=precision, method=args.method,
                                   shared_w=SW)
    g = api.reverse(rec, P, Y, layout="soa", shared_w=SW)
    off, h = rec.export_mesh()
    o = oracle.replay_grad(args.problem, wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"], off, h,
                           method=oracle_method(args), w=None if wl["w"] is None else np.asarray(SW.cpu().numpy(),
                                                                                                dtype=np.float64))
    a = np.concatenate([g["params_bar"].cpu().numpy().T, g["y0_bar"].cpu().numpy().T], 1)
    b = np.concatenate([o["params_bar"], o["y0_bar"]], 1)
    e = np.abs(a - b).max(1) / np.abs(b).max(1)
    rec.free()
    out = {"median": float(np.median(e)), "max": float(e.max()), "sample": m,
           "reference": "FP64 oracle replayed on the GPU's own mesh (normwise per trajectory)"}
    if args.problem in ("lorenz", "vdp"):
        # the achieved error against the converged gradient (FP64 oracle at rtol 1e-11 on its
        # own mesh): discretisation plus arithmetic, the quantity at which forms are matched
        fine = W.make(args.problem, m, seed=0)
        gf = oracle.solve_grad(fine["problem"], fine["params"], fine["y0"], fine["t0"], fine["t1"], fine["save_t"],
                               1e-12, 1e-14)
        c = np.concatenate([gf["params_bar"], gf["y0_bar"]], 1)
        ec = np.abs(a - c).max(1) / np.abs(c).max(1)
        comp = np.abs(a - c) / np.maximum(np.abs(c), 1e-30)
        out["vs_converged"] = {"median": float(np.median(ec)), "max": float(ec.max()),
                               "componentwise_median": float(np.median(comp)),
                               "componentwise_max": float(comp.max()),
                               "reference": "FP64 oracle at rtol 1e-12, atol 1e-14 on its own mesh (converged "
                                            "gradient); normwise per trajectory, and per component"}
    return out


def serving_measure(args):
    """The serving workload (uneven requests: problem ~ U{Lorenz, VdP, Robertson},
    n ~ 2^U[6, max], rtol ~ U{1e-6, 1e-8}, FP64, 64 GB record budget) through the
    continuous-batching server: capacity with all requests queued, then p50/p99
    latency under Poisson arrivals at 0.5 / 0.8 / 1.0 of that capacity, beside
    serial plain launches of the same stream."""
    from paper_2609_02876_gb300 import serve
    reqs = serve.c4_stream(args.serve_requests, seed=0, log2n=(6, args.serve_log2n_max))
    total = sum(r.n for r in reqs)
    serve.run_serial(reqs[:8])  # warm the kernels and allocators

    def server_run(rate):
        srv = serve.Server(slots=4, budget_bytes=64 << 30, max_pack=1 << 21)
        t = time.perf_counter()
        serve.run_stream(srv, reqs, rate=rate)
        dt = time.perf_counter() - t
        srv.close()
        assert all((r.status == 0).all() for r in reqs)
        lat = [r.latency for r in reqs]
        return dt, serve.latency_stats(lat), len(srv.batch_log)

    dt, stats, nb = server_run(None)
    cap_rps = len(reqs) / dt
    out = {"requests": len(reqs), "trajectories": total,
           "workload": f"{len(reqs)} requests, problem~U{{lorenz,vdp,robertson}}, n~2^U[6,{args.serve_log2n_max}], "
                       "rtol~U{1e-6,1e-8}, FP64, budget 64 GB, 4 slots",
           "capacity": {"requests_per_s": cap_rps, "trajectories_per_s": total / dt, "launches": nb}}
    for load in (0.5, 0.8, 1.0):
        dt, stats, nb = server_run(load * cap_rps)
        out[f"load_{load}"] = dict(stats, trajectories_per_s=total / dt, launches=nb)
    lat, dt = serve.run_serial(reqs)
    out["serial_all_queued"] = dict(serve.latency_stats(lat), trajectories_per_s=total / dt)
    lat, dt = serve.run_serial(reqs, rate=0.8 * cap_rps)
    out["serial_load_0.8"] = dict(serve.latency_stats(lat), trajectories_per_s=total / dt)
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    cores = os.cpu_count() or 1
    m = args.ref_sample
    wl = W.make(args.problem, m, rtol=args.rtol, seed=0)

    def step():
        g = oracle.solve_grad(wl["problem"], wl["params"], wl["y0"], wl["t0"], wl["t1"], wl["save_t"],
                              wl["rtol"], wl["atol"], nthreads=cores, method=oracle_method(args), w=wl["w"])
        assert g["ok"].all()

    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t
    v = m * args.steps / dt
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_of(args, m),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{m} trajectories of the {args.problem} workload per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def forward_measure(args, steps=5):
    """Forward-only solve (gs_solve, nothing recorded) on the paper's forward timing
    ensemble: Lorenz, rho evenly over [0, 21], sigma 10, beta 8/3, y0 (1, 0, 0),
    t in [0, 1], rtol 1e-6, atol 1e-9, solved to the final state, n = 2^24."""
    import torch
    from paper_2609_02876_gb300 import api
    n = args.forward_traj
    wl = W.make("lorenz_paper", n)
    P = torch.as_tensor(np.ascontiguousarray(wl["params"].T), device="cuda")
    Y = torch.as_tensor(np.ascontiguousarray(wl["y0"].T), device="cuda")
    uf = unit_flops("lorenz")
    res = {"workload": f"lorenz_paper n={n} t=[0,1] rtol=1e-6 atol=1e-9, final state only",
           "unit": "trajectories/s"}
    kms = np.zeros(2, np.float32)
    for prec in ("fp64", "fp32_mixed"):
        def run(**kw):
            return api.solve("lorenz", P, Y, wl["t0"], wl["t1"], [], wl["rtol"], wl["atol"], layout="soa",
                             want_saves=False, precision=prec, **kw)
        for _ in range(3):
            run()
        r = run(step_counts=True)
        assert (r["status"] == 0).all().item(), "trajectory failures in the forward workload"
        A_tot = int(r["step_counts"][1].to(torch.int64).sum().item())
        ms = []
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            run(kernel_ms=kms)
            ms.append(float(kms[0]))
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / steps
        ks = statistics.mean(ms) / 1e3
        ach = A_tot * uf["trial"] / ks / 1e12
        res[prec] = {"value": n / t, "us_per_traj": t / n * 1e6, "kernel_ms": ks * 1e3,
                     "attempted_steps_per_traj": A_tot / n, "achieved_tflops": ach,
                     "frac": ach / fp_peak_tflops(prec)}
    del P, Y
    return res


def forward_mode_measure(args, P, Y, wl, steps=3):
    """The gradient with respect to theta by forward mode (gs_forward_grad: one pass
    carrying the P unit directions) against the reverse sweep (gs_reverse) on the same
    record of the bench workload; the paper's comparison of the two modes."""
    import torch
    from paper_2609_02876_gb300 import api
    n = P.shape[1]
    rec, _, st = api.forward_record(args.problem, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                                    layout="soa", want_saves=False)

    def timed(f):
        for _ in range(2):
            f()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            f()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / steps

    t_fwd = timed(lambda: api.forward_grad(rec, P, Y, wrt=("params",), layout="soa"))
    t_rev = timed(lambda: api.reverse(rec, P, Y, layout="soa"))
    fw = api.forward_grad(rec, P, Y, wrt=("params",), layout="soa")["params_bar"]
    rv = api.reverse(rec, P, Y, layout="soa")["params_bar"]
    den = rv.abs().amax(0).clamp_min(1e-300)
    agree = ((fw - rv).abs().amax(0) / den).max().item()
    rec.free()
    return {"unit": "gradient trajectories/s (d loss / d theta, on a recorded mesh)",
            "forward_mode": n / t_fwd, "reverse_mode": n / t_rev, "forward_ms": t_fwd * 1e3,
            "reverse_ms": t_rev * 1e3, "max_rel_diff_forward_vs_reverse": agree}


def method_name(args):
    if args.method == "rosenbrock23":
        return "Rosenbrock23"
    if args.method == "verner7":
        return "Verner7"
    return "Rodas5P" if args.problem in STIFF else "Tsit5"


def config_of(args, n):
    wl = {"lorenz": "Lorenz-63 (sigma~U[8,12], rho~U[20,30], beta~U[2,3], y0~N((1,1,1),0.1^2 I), t in [0,1], "
                    "10 uniform saves)",
          "vdp": "Van der Pol (mu~U[0.5,2], y0~U[-2,2]^2, t in [0,10], 50 uniform saves)",
          "robertson": "Robertson (k=(0.04,3e7,1e4) x logU[0.9,1.1], y0=(1,0,0), t in [1e-5,1e5], 20 log saves)",
          "hires": "HIRES (12 rates x logU[0.9,1.1], standard y0, t in [0,321.8122], 10 uniform saves)",
          "lv_ude": "LV UDE (a~U[1,1.5], d~U[2,3], y0~U[0.5,2]^2, t in [0,5], 10 uniform saves, shared MLP "
                    "2-16-16-2 tanh, Glorot seed 0; grads also wrt the 354 shared weights)",
          "nrob": "Robertson neural RHS (k2 y2^2 -> MLP 3-16-16-1 tanh/softplus, FP64, Glorot seed 0; k1~U[0.04,0.06], "
                  "k3=1e4, y0=(1,0,0), t in [1e-5,1e5], 20 log saves; grads also wrt the 353 shared weights)",
          }[args.problem]
    method = method_name(args)
    atol = 1e-10 if args.problem in STIFF else args.rtol * 1e-2
    return {"workload": f"{wl}, {method} rtol={args.rtol:g} atol={atol:g}, {args.precision}, "
                        f"n={n} per GPU, loss=sum_s ||y(t_s)||^2, grads wrt theta and y0",
            "n_per_gpu": n, "problem": args.problem, "precision": args.precision, "rtol": args.rtol,
            "l2": "inputs and record larger than L2 (no flush)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gradsolve", choices=["gradsolve", "reference"])
    ap.add_argument("--problem", default="lorenz", choices=["lorenz", "vdp", "robertson", "hires", "lv_ude", "nrob"])
    ap.add_argument("--traj", type=int, default=1 << 24, help="trajectories per GPU")
    ap.add_argument("--rtol", type=float, default=1e-6)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_mixed"])
    ap.add_argument("--method", default=None, choices=["rodas5p", "rosenbrock23", "verner7"],
                    help="method (default: Rodas5P for the stiff problems, Tsit5 otherwise; Rosenbrock23 for "
                         "stiff ones, Verner7 for Lorenz and Van der Pol on request)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=1 << 15)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-forward", action="store_true")
    ap.add_argument("--no-forward-mode", action="store_true")
    ap.add_argument("--forward-traj", type=int, default=1 << 24)
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-log2n-max", type=int, default=18)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2609_02876_gb300 import api, build
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    n = args.traj
    if args.problem == "lv_ude":
        args.precision = "fp32_mixed"  # FP32 network and state, FP64 step control
    wl = W.make(args.problem, n, rtol=args.rtol, seed=rank)
    P = torch.as_tensor(np.ascontiguousarray(wl["params"].T), device="cuda")
    Y = torch.as_tensor(np.ascontiguousarray(wl["y0"].T), device="cuda")
    SW = None if wl["w"] is None else torch.as_tensor(np.asarray(wl["w"], dtype=np.float32), device="cuda")
    d, Pn, _, _ = api.problem_info(args.problem)
    out = {"loss": torch.empty(n, dtype=torch.float64, device="cuda"),
           "params_bar": torch.empty((Pn, n), dtype=torch.float64, device="cuda"),
           "y0_bar": torch.empty((d, n), dtype=torch.float64, device="cuda"),
           "status": torch.empty(n, dtype=torch.int32, device="cuda")}
    kms = np.zeros(2, np.float32)
    rinfo = np.zeros(2, np.int32)  # checkpoint interval k, stored stages

    def step(kernel_ms=None, counts=False):
        return api.solve_grad(args.problem, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                              layout="soa", out=out, precision=args.precision, kernel_ms=kernel_ms,
                              step_counts=counts, method=args.method, shared_w=SW, record_info=rinfo)

    for _ in range(args.warmup):
        step()
    r = step(counts=True)
    assert (out["status"] == 0).all().item(), "trajectory failures in the benchmark workload"
    sc = r["step_counts"].to(torch.int64).sum(1).tolist()
    S_tot, A_tot = sc[0], sc[1]

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    fwd_ms, rev_ms = [], []
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step(kernel_ms=kms)
        fwd_ms.append(float(kms[0]))
        rev_ms.append(float(kms[1]))
    e1.record()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    t = e0.elapsed_time(e1) / 1e3
    if ws > 1:
        tt = torch.tensor([t], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t = tt.item()
    value = ws * n * args.steps / t

    # end to end through the public API: gs_solve_grad_host reads the inputs from
    # pinned host memory and writes the results back to it, with the copies of
    # one chunk overlapping the solve of the next
    hP = torch.from_numpy(np.ascontiguousarray(wl["params"].T)).pin_memory()
    hY = torch.from_numpy(np.ascontiguousarray(wl["y0"].T)).pin_memory()
    hout = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
    ke = max(1, min(args.steps, 3))

    def host_step():
        api.solve_grad_host(args.problem, hP, hY, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                            shared_w=SW, out=hout, precision=args.precision, method=args.method, check=False)

    host_step()  # warm-up (staging buffers)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        host_step()
    te = time.perf_counter() - t0
    barrier()
    h2d = (hP.numel() + hY.numel()) * 8
    d2h = sum(v.numel() * v.element_size() for v in hout.values())
    e2e = {"value": ws * n * ke / te, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # roofline of the dominant kernel (the reverse sweep), algorithmic flops / event-timed duration
    uf = unit_flops(args.problem, args.method)
    n_side = n * (len(wl["save_t"]) - 1)  # saves strictly inside a step (the last one sits on t1)
    stages = bool(rinfo[1])
    if stages:
        # stored stages: the record also runs the side steps (trial code) and the reverse
        # sweep only propagates cotangents through the stored stages
        rev_flops = (S_tot + n_side) * (uf["vjp_unit"] - uf["stage_fwd"])
        fwd_flops = (A_tot + n_side) * uf["trial"]
    else:
        rev_flops = (S_tot + n_side) * uf["vjp_unit"]
        fwd_flops = A_tot * uf["trial"]
    layout = "stages" if stages else "compact"
    rev_s = statistics.mean(rev_ms) / 1e3
    fwd_s = statistics.mean(fwd_ms) / 1e3
    peak = fp_peak_tflops(args.precision)
    dominant = "reverse" if rev_s >= fwd_s else "record"
    ach = (rev_flops / rev_s if dominant == "reverse" else fwd_flops / fwd_s) / 1e12
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": config_of(args, n),
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "traffic": (TRAFFIC_PER_STEP[(args.problem, args.precision, dominant, layout)] * S_tot
                                     if (args.problem, args.precision, dominant, layout) in TRAFFIC_PER_STEP
                                     and args.method is None else None),
                         "kernel": f"{dominant}_kernel<{method_name(args)}>",
                         "peak_source": "derived: 152 SMs x FMA lanes/clk/SM x 2 x 2070 MHz"},
            "kernels_ms": {"record": statistics.mean(fwd_ms), "reverse": statistics.mean(rev_ms)},
            "work": {"accepted_steps": S_tot, "attempted_steps": A_tot, "record_tflops": fwd_flops / fwd_s / 1e12,
                     "record_layout": {"k": int(rinfo[0]), "stored_stages": stages},
                     "record_dram_gbs": (TRAFFIC_PER_STEP[(args.problem, args.precision, "record", layout)] * S_tot
                                         / fwd_s / 1e9
                                         if (args.problem, args.precision, "record", layout) in TRAFFIC_PER_STEP
                                         and args.method is None else None),
                     "reverse_dram_gbs": (TRAFFIC_PER_STEP[(args.problem, args.precision, "reverse", layout)] * S_tot
                                          / rev_s / 1e9
                                          if (args.problem, args.precision, "reverse", layout) in TRAFFIC_PER_STEP
                                          and args.method is None else None),
                     "reverse_tflops": rev_flops / rev_s / 1e12},
            "e2e": e2e, "gpu_launches": (3 if args.problem in ("lv_ude", "nrob") else 2) * args.steps, "clocks": clocks}
    if rank == 0:
        line["accuracy"] = accuracy_sample(args, args.precision)
    if rank == 0 and ws == 1 and args.precision == "fp64" and args.problem in ("lorenz", "vdp") \
            and not args.no_mixed:
        # the FP32-mixed form on the same workload and GPU: throughput and its error vs the FP64 oracle
        for _ in range(2):
            api.solve_grad(args.problem, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                           layout="soa", out=out, precision="fp32_mixed")
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            api.solve_grad(args.problem, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                           layout="soa", out=out, precision="fp32_mixed")
        e1.record()
        torch.cuda.synchronize()
        tm = e0.elapsed_time(e1) / 1e3
        line["fp32_mixed"] = {"value": n * args.steps / tm, "unit": UNIT, "ms_per_step": tm / args.steps * 1e3,
                              "dtype": "f32 stages/adjoint + f64 control",
                              "accuracy": accuracy_sample(args, "fp32_mixed")}
    if rank == 0 and ws == 1 and not args.no_forward_mode and args.problem in ("lorenz", "vdp", "robertson"):
        line["forward_vs_reverse_mode"] = forward_mode_measure(args, P, Y, wl)
    if rank == 0 and ws == 1 and not args.no_forward:
        line["forward_only"] = forward_measure(args)
    if rank == 0 and ws == 1 and not args.no_serve:
        line["serving"] = serving_measure(args)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
