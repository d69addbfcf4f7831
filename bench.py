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

Besides the timed headline the line carries, on rank 0 of a one-GPU run:
the gradient error of a random sample of the timed run's own outputs against
the FP64 oracle replayed on the same trajectories' GPU mesh, the mesh's
agreement with the oracle's own record, the FP64-control and FP32-mixed forms
(both step controls) at matched error, the forward-only solve, forward against
reverse mode, the other configurations (Lorenz n = 1024, Van der Pol,
Robertson and HIRES with Rodas5P, the LV UDE), the serving stream and the
oracle's CPU rate. Every roofline fraction is taken against the FMA rate
measured on the same GPU at the start of the run (gs_measure_fma_peak).

Launch: python bench.py [--gpus N --steps K --warmup W] on one GPU, or under
torchrun (one rank per GPU, each rank its own shard: weak scaling).
`--impl reference` times the FP64 CPU oracle on the host cores instead.
`--profile-case {solve_grad,forward_only,jvp}` runs one workload four times
(three warm-up calls, then the one to capture with ncu) and prints no JSON.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
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
# the same FP64 workload, stored-stage layout (Lorenz: 45.15 accepted steps per
# trajectory; Robertson: 101243901 accepted steps in all); a launch's traffic grows
# in proportion to its accepted steps. The Lorenz reverse sweep's writes are its
# register spills (the kernel is capped at 96 registers).
TRAFFIC_PER_STEP = {("lorenz", "fp64", "reverse", "stages"): (14935465472 + 328079616) / (45.15 * 2 ** 20),
                    ("lorenz", "fp64", "record", "stages"): (291875328 + 9850115584) / (45.15 * 2 ** 20),
                    ("robertson", "fp64", "reverse", "stages"): (49664537600 + 67086336) / 101243901,
                    ("robertson", "fp64", "record", "stages"): (2908891648 + 67400810240) / 101243901}

# Nominal FMA lanes per SM per clock of this part (FP64 at 1/64 of FP32), for the
# nominal peak printed beside the measured one.
NOMINAL_LANES = {"fp64": 2, "fp32_mixed": 128}


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


def measure_peaks():
    """FMA throughput of this GPU's FP64 and FP32 pipes (gs_measure_fma_peak), TFLOP/s."""
    import ctypes as C

    from paper_2609_02876_gb300 import _native as N
    out = {}
    for kind, name in ((0, "fp64_fma"), (1, "fp32_fma"), (2, "fp32x2_fma")):
        v = C.c_double(0.0)
        rc = N.lib().gs_measure_fma_peak(kind, C.byref(v))
        out[name] = v.value if rc == N.GS_OK else None
    return out


def peak_of(precision, peaks):
    """The measured denominator of a form: FP64 FMA, or the faster FP32 FMA form."""
    if precision == "fp64":
        return peaks["fp64_fma"]
    return max(peaks["fp32_fma"] or 0.0, peaks["fp32x2_fma"] or 0.0)


def nominal_peak(precision, sm_mhz=2070.0):
    return 152 * NOMINAL_LANES[precision] * 2 * sm_mhz * 1e6 / 1e12


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


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform)."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for ln in r.stdout.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def oracle_method(method):
    import oracle
    return {"rosenbrock23": oracle.METHOD_ROSENBROCK23, "verner7": oracle.METHOD_VERNER7}.get(method,
                                                                                         oracle.METHOD_AUTO)


def cpu_baseline(args, budget_s=12.0):
    """The FP64 oracle (record + replay gradient), as it stands, on the host cores,
    over a bounded sample of the same workload."""
    import oracle
    cores = os.cpu_count() or 1
    om = oracle_method(args.method)
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
    return {"value": m / dt, "unit": UNIT, "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"first {m} trajectories of the same {args.problem} workload (seed 0), record + replay "
                      f"gradient, {dt:.1f} s on {cores} threads"}


def _normwise(a, b):
    return np.abs(a - b).max(1) / np.maximum(np.abs(b).max(1), 1e-300)


def sample_accuracy(problem, wl, out, precision, method=None, control="fast", m=4096, seed=12345,
                    converged=False, shared_w=None):
    """Gradient error of the timed run's own outputs (`out`, SoA device tensors of
    the whole ensemble) at m trajectories drawn at random from it, against the FP64
    oracle replayed on those trajectories' GPU mesh (recorded again for the sample:
    trajectories are independent, so it is the mesh of the timed run, which the
    bit-identity of the sample's own GPU gradient confirms); plus the mesh's
    agreement with the oracle's own record of the same trajectories, and (Lorenz,
    Van der Pol) the error against the converged gradient."""
    import torch

    import oracle
    from paper_2609_02876_gb300 import api
    n = wl["params"].shape[0]
    idx = np.sort(np.random.default_rng(seed).choice(n, size=min(m, n), replace=False))
    sp, sy = wl["params"][idx], wl["y0"][idx]
    P = torch.as_tensor(np.ascontiguousarray(sp.T), device="cuda")
    Y = torch.as_tensor(np.ascontiguousarray(sy.T), device="cuda")
    rec, _, _ = api.forward_record(problem, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                                   layout="soa", want_saves=False, precision=precision, method=method,
                                   shared_w=shared_w, control=control)
    g = api.reverse(rec, P, Y, layout="soa", shared_w=shared_w)
    off, h = rec.export_mesh()
    rec.free()
    w64 = None if wl["w"] is None else np.asarray(shared_w.cpu().numpy(), dtype=np.float64)
    om = oracle_method(method)
    o = oracle.replay_grad(problem, sp, sy, wl["t0"], wl["t1"], wl["save_t"], off, h, method=om, w=w64)
    big = np.concatenate([out["params_bar"][:, idx].cpu().numpy().T, out["y0_bar"][:, idx].cpu().numpy().T], 1)
    small = np.concatenate([g["params_bar"].cpu().numpy().T, g["y0_bar"].cpu().numpy().T], 1)
    ref = np.concatenate([o["params_bar"], o["y0_bar"]], 1)
    e = _normwise(big, ref)
    res = {"median": float(np.median(e)), "max": float(e.max()), "sample": int(idx.size),
           "sample_bit_identical_to_timed_run": bool(np.array_equal(big, small)),
           "reference": f"FP64 oracle replayed on the GPU mesh of {idx.size} trajectories drawn at random from the "
                        "timed run (normwise per trajectory vector of (theta_bar, y0_bar))"}
    if shared_w is not None and "shared_w_bar" in g:
        wb, wr = g["shared_w_bar"].cpu().numpy().astype(np.float64), o["w_bar"]
        res["shared_w_bar_rel_err"] = float(np.abs(wb - wr).max() / np.abs(wr).max())
    orec = oracle.record(problem, sp, sy, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"], method=om,
                         w=w64, want_saves=False)
    same = np.diff(off) == orec["S"]
    worst = 0.0
    for k in np.nonzero(same)[0]:
        a = h[off[k]:off[k + 1]]
        b = orec["h"][orec["offsets"][k]:orec["offsets"][k + 1]]
        if a.size > 1:
            worst = max(worst, float((np.abs(a - b) / b)[:-1].max()))
    res["mesh_vs_oracle_record"] = {"equal_step_count_fraction": float(same.mean()),
                                    "max_rel_h_diff_equal_counts": worst,
                                    "steps_per_traj_gpu": float(np.diff(off).mean()),
                                    "steps_per_traj_oracle": float(orec["S"].mean())}
    if converged and problem in ("lorenz", "vdp"):
        fine = oracle.solve_grad(problem, sp, sy, wl["t0"], wl["t1"], wl["save_t"], 1e-12, 1e-14)
        c = np.concatenate([fine["params_bar"], fine["y0_bar"]], 1)
        ec = _normwise(big, c)
        comp = np.abs(big - c) / np.maximum(np.abs(c), 1e-30)
        res["vs_converged"] = {"median": float(np.median(ec)), "max": float(ec.max()),
                               "componentwise_median": float(np.median(comp)),
                               "componentwise_max": float(comp.max()),
                               "reference": "FP64 oracle at rtol 1e-12, atol 1e-14 on its own mesh (converged "
                                            "gradient); normwise per trajectory, and per component"}
    return res


class Form:
    """One (problem, n, precision, method, control) ensemble resident on the GPU,
    stepped through api.solve_grad."""

    def __init__(self, problem, n, rtol=None, precision="fp64", method=None, control="fast", seed=0):
        import torch

        from paper_2609_02876_gb300 import api
        self.api = api
        self.problem, self.n, self.precision, self.method, self.control = problem, n, precision, method, control
        self.wl = W.make(problem, n, rtol=rtol, seed=seed)
        wl = self.wl
        self.P = torch.as_tensor(np.ascontiguousarray(wl["params"].T), device="cuda")
        self.Y = torch.as_tensor(np.ascontiguousarray(wl["y0"].T), device="cuda")
        self.SW = None if wl["w"] is None else torch.as_tensor(np.asarray(wl["w"], dtype=np.float32), device="cuda")
        d, Pn, _, _ = api.problem_info(problem)
        self.out = {"loss": torch.empty(n, dtype=torch.float64, device="cuda"),
                    "params_bar": torch.empty((Pn, n), dtype=torch.float64, device="cuda"),
                    "y0_bar": torch.empty((d, n), dtype=torch.float64, device="cuda"),
                    "status": torch.empty(n, dtype=torch.int32, device="cuda")}
        self.kms = np.zeros(2, np.float32)
        self.rinfo = np.zeros(2, np.int32)

    def step(self, timed=False, counts=False):
        wl = self.wl
        return self.api.solve_grad(self.problem, self.P, self.Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"],
                                   wl["atol"], layout="soa", out=self.out, precision=self.precision,
                                   kernel_ms=self.kms if timed else None, step_counts=counts, method=self.method,
                                   shared_w=self.SW, record_info=self.rinfo, control=self.control)

    def counts(self):
        import torch
        r = self.step(counts=True)
        assert (self.out["status"] == 0).all().item(), f"trajectory failures in the {self.problem} workload"
        sc = r["step_counts"].to(torch.int64).sum(1).tolist()
        self.S_tot, self.A_tot = sc[0], sc[1]

    def timed(self, steps, barrier=lambda: None):
        """Times `steps` calls with CUDA events around all of them and around each
        kernel; returns seconds per step."""
        import torch
        rec_ms, rev_ms = [], []
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            self.step(timed=True)
            rec_ms.append(float(self.kms[0]))
            rev_ms.append(float(self.kms[1]))
        e1.record()
        torch.cuda.synchronize()
        barrier()
        self.rec_s = statistics.mean(rec_ms) / 1e3
        self.rev_s = statistics.mean(rev_ms) / 1e3
        return e0.elapsed_time(e1) / 1e3 / steps

    def roofline(self, peaks):
        """ALU roofline of the dominant kernel: algorithmic flops / event-timed duration."""
        uf = unit_flops(self.problem, self.method)
        n_side = self.n * (len(self.wl["save_t"]) - 1)  # saves strictly inside a step (the last sits on t1)
        stages = bool(self.rinfo[1])
        if stages:
            # stored stages: the record also runs the side steps (trial code) and the reverse
            # sweep only propagates cotangents through the stored stages
            rev_flops = (self.S_tot + n_side) * (uf["vjp_unit"] - uf["stage_fwd"])
            fwd_flops = (self.A_tot + n_side) * uf["trial"]
        else:
            rev_flops = (self.S_tot + n_side) * uf["vjp_unit"]
            fwd_flops = self.A_tot * uf["trial"]
        layout = "stages" if stages else "compact"
        dominant = "reverse" if self.rev_s >= self.rec_s else "record"
        ach = (rev_flops / self.rev_s if dominant == "reverse" else fwd_flops / self.rec_s) / 1e12
        peak = peak_of(self.precision, peaks)
        key = (self.problem, self.precision, dominant, layout)
        traffic = (TRAFFIC_PER_STEP[key] * self.S_tot if key in TRAFFIC_PER_STEP and self.method is None
                   and self.control == "fast" else None)
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": traffic, "kernel": f"{dominant}_kernel<{method_name(self.problem, self.method)}>",
                "peak_source": ("measured on this GPU at the start of the run (gs_measure_fma_peak: "
                                + ("FP64 FMA" if self.precision == "fp64" else "the faster of FP32 and FP32x2 FMA")
                                + ")"),
                "peak_nominal": nominal_peak(self.precision),
                "frac_of_nominal": ach / nominal_peak(self.precision)}
        work = {"accepted_steps": self.S_tot, "attempted_steps": self.A_tot,
                "record_tflops": fwd_flops / self.rec_s / 1e12, "reverse_tflops": rev_flops / self.rev_s / 1e12,
                "record_frac": fwd_flops / self.rec_s / 1e12 / peak,
                "reverse_frac": rev_flops / self.rev_s / 1e12 / peak,
                "record_layout": {"k": int(self.rinfo[0]), "stored_stages": stages}}
        for kern, secs in (("record", self.rec_s), ("reverse", self.rev_s)):
            k2 = (self.problem, self.precision, kern, layout)
            work[f"{kern}_dram_gbs"] = (TRAFFIC_PER_STEP[k2] * self.S_tot / secs / 1e9
                                        if k2 in TRAFFIC_PER_STEP and self.method is None
                                        and self.control == "fast" else None)
        return roof, work

    def free(self):
        for k in ("P", "Y", "out", "SW"):
            if hasattr(self, k):
                delattr(self, k)


def leg(problem, n, peaks, precision="fp64", method=None, control="fast", steps=3, warmup=2, rtol=None,
        acc_m=1024, converged=False):
    """A secondary configuration: throughput, kernel times, roofline and sampled accuracy."""
    f = Form(problem, n, rtol=rtol, precision=precision, method=method, control=control)
    for _ in range(warmup):
        f.step()
    f.counts()
    t = f.timed(steps)
    roof, work = f.roofline(peaks)
    res = {"workload": config_of(problem, f.wl["rtol"], precision, n, method)["workload"],
           "value": n / t, "unit": UNIT, "ms_per_step": t * 1e3,
           "kernels_ms": {"record": f.rec_s * 1e3, "reverse": f.rev_s * 1e3},
           "control": control, "roofline": roof, "work": work,
           "accuracy": sample_accuracy(problem, f.wl, f.out, precision, method, control, m=acc_m,
                                       converged=converged, shared_w=f.SW)}
    f.free()
    return res


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
        srv = serve.Server(slots=4, budget_bytes=64 << 30, max_pack=1 << 21, max_chunk=args.serve_chunk)
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
                       f"rtol~U{{1e-6,1e-8}}, FP64, budget 64 GB, 4 slots, chunks of at most {args.serve_chunk} "
                       "trajectories",
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
                              wl["rtol"], wl["atol"], nthreads=cores, method=oracle_method(args.method), w=wl["w"])
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
            "config": config_of(args.problem, args.rtol, args.precision, m, args.method),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
                             "sample": f"{m} trajectories of the {args.problem} workload per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def forward_measure(args, peaks, steps=5):
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
                     "frac": ach / peak_of(prec, peaks)}
    del P, Y
    return res


def launches_per_step(problem, precision, k, wl):
    """Kernels one gs_solve_grad call launches: the starting-step pass, the record, the
    t1-save pass (FP64, no shared weights, k = 1, last save time t1), the reverse sweep,
    and for shared-weight problems the weight-gradient reduction."""
    weights = problem in ("lv_ude", "nrob")
    st = np.asarray(wl["save_t"], dtype=np.float64)
    t1_pass = (precision == "fp64" and not weights and k == 1 and st.size > 0
               and st[-1].tobytes() == np.float64(wl["t1"]).tobytes())
    return 3 + int(t1_pass) + int(weights)


def record_memory_measure():
    """Device memory of the record (gs_record_bytes) for the paper's memory case, the
    neural Robertson at B = 128 trajectories (Rodas5P, compact record), and for a 2^20
    Lorenz ensemble in both record layouts (compact and stored stages)."""
    import torch
    from paper_2609_02876_gb300 import api
    out = {}
    for key, name, n, opts in (("nrob_B128", "nrob", 128, {}),
                               ("lorenz_2^20_compact", "lorenz", 1 << 20, {"ckpt_k": 1}),
                               ("lorenz_2^20_stored_stages", "lorenz", 1 << 20, {"ckpt_k": 1, "record_stages": True})):
        wl = W.make(name, n)
        P = torch.as_tensor(np.ascontiguousarray(wl["params"].T), device="cuda")
        Y = torch.as_tensor(np.ascontiguousarray(wl["y0"].T), device="cuda")
        w = None if wl["w"] is None else torch.as_tensor(np.asarray(wl["w"], dtype=np.float32), device="cuda")
        rec, _, _ = api.forward_record(name, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                                       layout="soa", shared_w=w, want_saves=False, **opts)
        st = rec.stats()
        out[key] = {"n": n, "record_bytes": rec.bytes(), "accepted_steps": st["accepted"],
                    "bytes_per_accepted_step": rec.bytes() / max(st["accepted"], 1)}
        rec.free()
        del P, Y
        torch.cuda.empty_cache()
    return out


def forward_mode_measure(problem, P, Y, wl, steps=3):
    """The gradient with respect to theta by forward mode (gs_forward_grad: one pass
    carrying the P unit directions) against the reverse sweep (gs_reverse) on the same
    record of the bench workload; the paper's comparison of the two modes."""
    import torch
    from paper_2609_02876_gb300 import api
    n = P.shape[1]
    rec, _, st = api.forward_record(problem, P, Y, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
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


def method_name(problem, method):
    if method == "rosenbrock23":
        return "Rosenbrock23"
    if method == "verner7":
        return "Verner7"
    return "Rodas5P" if problem in STIFF else "Tsit5"


def config_of(problem, rtol, precision, n, method=None):
    wl = {"lorenz": "Lorenz-63 (sigma~U[8,12], rho~U[20,30], beta~U[2,3], y0~N((1,1,1),0.1^2 I), t in [0,1], "
                    "10 uniform saves)",
          "vdp": "Van der Pol (mu~U[0.5,2], y0~U[-2,2]^2, t in [0,10], 50 uniform saves)",
          "robertson": "Robertson (k=(0.04,3e7,1e4) x logU[0.9,1.1], y0=(1,0,0), t in [1e-5,1e5], 20 log saves)",
          "hires": "HIRES (12 rates x logU[0.9,1.1], standard y0, t in [0,321.8122], 10 uniform saves)",
          "lv_ude": "LV UDE (a~U[1,1.5], d~U[2,3], y0~U[0.5,2]^2, t in [0,5], 10 uniform saves, shared MLP "
                    "2-16-16-2 tanh, Glorot seed 0; grads also wrt the 354 shared weights)",
          "nrob": "Robertson neural RHS (k2 y2^2 -> MLP 3-16-16-1 tanh/softplus, FP64, Glorot seed 0; k1~U[0.04,0.06], "
                  "k3=1e4, y0=(1,0,0), t in [1e-5,1e5], 20 log saves; grads also wrt the 353 shared weights)",
          }[problem]
    if rtol is None:
        rtol = 1e-6
    atol = 1e-10 if problem in STIFF else rtol * 1e-2
    return {"workload": f"{wl}, {method_name(problem, method)} rtol={rtol:g} atol={atol:g}, {precision}, "
                        f"n={n} per GPU, loss=sum_s ||y(t_s)||^2, grads wrt theta and y0",
            "n_per_gpu": n, "problem": problem, "precision": precision, "rtol": rtol,
            "l2": "inputs and record larger than L2 (no flush)"}


def profile_case(args):
    """One workload run four times (three warm-up calls, then the one an ncu
    capture selects with -s / -c by kernel name); prints one line, no JSON."""
    import torch

    from paper_2609_02876_gb300 import api
    wl = W.make(args.problem, args.traj, rtol=args.rtol)
    P = torch.as_tensor(np.ascontiguousarray(wl["params"].T), device="cuda")
    Y = torch.as_tensor(np.ascontiguousarray(wl["y0"].T), device="cuda")
    SW = None if wl["w"] is None else torch.as_tensor(np.asarray(wl["w"], dtype=np.float32), device="cuda")
    common = (wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"])
    kw = dict(layout="soa", precision=args.precision, shared_w=SW, method=args.method, control=args.control)
    if args.profile_case == "solve_grad":
        def run():
            return api.solve_grad(args.problem, P, Y, *common, **kw)
    elif args.profile_case == "forward_only":
        def run():
            return api.solve(args.problem, P, Y, *common, **kw)
    else:
        rec, _, _ = api.forward_record(args.problem, P, Y, *common, layout="soa", want_saves=False,
                                       method=args.method)

        def run():
            return api.forward_grad(rec, P, Y, wrt=("params",), layout="soa")
    for _ in range(4):
        run()
    torch.cuda.synchronize()
    print(f"{args.profile_case} {args.problem} n={args.traj} {args.precision} {args.control}: ok", flush=True)
    return 0


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
    ap.add_argument("--control", default="fast", choices=["fast", "fp64"],
                    help="step-size control evaluation (GS_CONTROL_FAST or GS_CONTROL_FP64)")
    ap.add_argument("--method", default=None, choices=["rodas5p", "rosenbrock23", "verner7"],
                    help="method (default: Rodas5P for the stiff problems, Tsit5 otherwise; Rosenbrock23 for "
                         "stiff ones, Verner7 for Lorenz and Van der Pol on request)")
    ap.add_argument("--profile-case", default=None, choices=["solve_grad", "forward_only", "jvp"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=1 << 15)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-forward", action="store_true")
    ap.add_argument("--no-forward-mode", action="store_true")
    ap.add_argument("--no-legs", action="store_true", help="skip the other configurations")
    ap.add_argument("--forward-traj", type=int, default=1 << 24)
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-log2n-max", type=int, default=20)
    ap.add_argument("--serve-chunk", type=int, default=1 << 16)
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
    if args.problem == "lv_ude":
        args.precision = "fp32_mixed"  # FP32 network and state, FP64 step control
    if args.profile_case:
        return profile_case(args)
    peaks = measure_peaks()
    n = args.traj
    f = Form(args.problem, n, rtol=args.rtol, precision=args.precision, method=args.method, control=args.control,
             seed=rank)
    wl = f.wl
    for _ in range(args.warmup):
        f.step()
    f.counts()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    t = f.timed(args.steps, barrier) * args.steps
    clocks = sampler.stop()
    if ws > 1:
        tt = torch.tensor([t], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t = tt.item()
    value = ws * n * args.steps / t
    roof, work = f.roofline(peaks)

    # end to end through the public API: gs_solve_grad_host reads the inputs from
    # pinned host memory and writes the results back to it, with the copies of
    # one chunk overlapping the solve of the next; timed over as many calls as
    # the device-resident steps
    hP = torch.from_numpy(np.ascontiguousarray(wl["params"].T)).pin_memory()
    hY = torch.from_numpy(np.ascontiguousarray(wl["y0"].T)).pin_memory()
    hout = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in f.out.items()}

    def host_step():
        api.solve_grad_host(args.problem, hP, hY, wl["t0"], wl["t1"], wl["save_t"], wl["rtol"], wl["atol"],
                            shared_w=f.SW, out=hout, precision=args.precision, method=args.method,
                            control=args.control, check=False)

    host_step()  # warm-up (staging buffers)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        host_step()
    te = time.perf_counter() - t0
    barrier()
    if ws > 1:
        tt = torch.tensor([te], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        te = tt.item()
    h2d = (hP.numel() + hY.numel()) * 8
    d2h = sum(v.numel() * v.element_size() for v in hout.values())
    e2e = {"value": ws * n * args.steps / te, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "calls": args.steps}
    del hP, hY, hout

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": dict(config_of(args.problem, args.rtol, args.precision, n, args.method), control=args.control),
            "roofline": roof, "kernels_ms": {"record": f.rec_s * 1e3, "reverse": f.rev_s * 1e3},
            "work": work, "peaks_measured": peaks,
            "e2e": e2e, "gpu_launches": launches_per_step(args.problem, args.precision, int(f.rinfo[0]),
                                                          f.wl) * args.steps, "clocks": clocks}
    solo = rank == 0 and ws == 1
    if rank == 0:
        line["accuracy"] = sample_accuracy(args.problem, wl, f.out, args.precision, args.method, args.control,
                                           converged=True, shared_w=f.SW)
    f.free()
    torch.cuda.empty_cache()
    if solo and args.precision == "fp64" and args.problem in ("lorenz", "vdp") and args.method is None \
            and not args.no_mixed:
        # the same workload with the other step control, and in the FP32-mixed form with
        # both controls: throughput, kernel roofline and error, at matched gradient error
        other = "fp64" if args.control == "fast" else "fast"
        forms = {f"fp64_control_{other}": ("fp64", other), "fp32_mixed": ("fp32_mixed", "fast"),
                 "fp32_mixed_control_fp64": ("fp32_mixed", "fp64")}
        for key, (prec, ctrl) in forms.items():
            g = Form(args.problem, n, rtol=args.rtol, precision=prec, control=ctrl)
            for _ in range(2):
                g.step()
            g.counts()
            tm = g.timed(args.steps)
            r2, w2 = g.roofline(peaks)
            line[key] = {"value": n / tm, "unit": UNIT, "ms_per_step": tm * 1e3,
                         "dtype": ("f32 stages/adjoint + f64 t, h" if prec == "fp32_mixed" else "f64"),
                         "control": ctrl, "kernels_ms": {"record": g.rec_s * 1e3, "reverse": g.rev_s * 1e3},
                         "roofline": r2, "work": w2,
                         "accuracy": sample_accuracy(args.problem, g.wl, g.out, prec, None, ctrl, converged=True)}
            g.free()
            torch.cuda.empty_cache()
    if solo and not args.no_forward_mode and args.problem in ("lorenz", "vdp", "robertson"):
        fm = Form(args.problem, min(n, 1 << 22), rtol=args.rtol)
        line["forward_vs_reverse_mode"] = forward_mode_measure(args.problem, fm.P, fm.Y, fm.wl)
        line["forward_vs_reverse_mode"]["n"] = fm.n
        fm.free()
        torch.cuda.empty_cache()
    if solo and not args.no_forward:
        line["forward_only"] = forward_measure(args, peaks)
        torch.cuda.empty_cache()
    if solo and not args.no_legs:
        line["record_memory"] = record_memory_measure()
    if solo and not args.no_legs:
        # the other configurations: Lorenz at the small size, the Van der Pol part of the
        # non-stiff sweep, the stiff kinetics with Rodas5P at their largest sizes, the LV UDE
        legs = {"lorenz_n1024": dict(problem="lorenz", n=1024, acc_m=1024),
                "vdp_n2^22": dict(problem="vdp", n=1 << 22, converged=True),
                "robertson_n2^20": dict(problem="robertson", n=1 << 20),
                "hires_n2^18": dict(problem="hires", n=1 << 18),
                "lv_ude_n2^18": dict(problem="lv_ude", n=1 << 18, precision="fp32_mixed")}
        line["configs"] = {}
        for key, kw in legs.items():
            line["configs"][key] = leg(peaks=peaks, **kw)
            torch.cuda.empty_cache()
    if solo and not args.no_serve:
        line["serving"] = serving_measure(args)
    if solo and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
