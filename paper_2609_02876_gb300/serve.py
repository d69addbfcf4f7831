"""Continuous-batching request server for gradient requests (one GPU).

A request is one ensemble: (problem, params (n, P), y0 (n, d), rtol), host
arrays. The server keeps `slots` solve contexts (each its own device
workspace and CUDA stream, driven by one host thread). Whenever a slot is
free it takes the oldest waiting request and packs every other waiting
request with the same (problem, rtol) behind it, up to `max_pack`
trajectories, into ONE launch of the persistent record + reverse kernels;
trajectories are independent, so each request's results are exactly those of
solving it alone (tested). A batch is admitted only if the estimated record
footprint of all batches in flight stays within `budget_bytes`; batches on
different slots overlap on the device. Latency = completion - arrival.

Only argument marshalling and scheduling live here; every step of the
solve runs in libgradsolve's kernels.
"""
from __future__ import annotations

import collections
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import api
from . import workloads as W

# Expected accepted steps per trajectory at rtol 1e-6 (the record-footprint
# estimate scales it by (1e-6 / rtol)^(1/5), the order-5 step-count law).
_STEPS_1E6 = {"lorenz": 48, "vdp": 100, "robertson": 100, "hires": 200, "lv_ude": 34}


def record_footprint(problem: str, n: int, rtol: float) -> int:
    """Estimated device bytes of the record of n trajectories (k = 1 layout:
    8 doubles per accepted step incl. the segment header, x1.25 margin)."""
    d, P, _, _ = api.problem_info(problem)
    steps = _STEPS_1E6[problem] * (1e-6 / rtol) ** 0.2
    seg = 8 * (((2 + d + 1) + 1) & ~1)
    return int(1.25 * n * steps * seg + n * (8 + 12 + 8 * d))


@dataclass
class Request:
    rid: int
    problem: str
    params: np.ndarray
    y0: np.ndarray
    rtol: float
    arrival: float = 0.0  # seconds on the server clock
    loss: np.ndarray | None = None
    params_bar: np.ndarray | None = None
    y0_bar: np.ndarray | None = None
    status: np.ndarray | None = None
    t_start: float = math.nan
    t_done: float = math.nan
    batch: int = -1
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def n(self) -> int:
        return self.params.shape[0]

    @property
    def key(self):
        return (self.problem, float(self.rtol))

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


def _spec(problem):
    """Time span, save times and atol rule of a problem's workload."""
    wl = W.make(problem, 1)
    atol_ratio = None if problem in ("robertson", "hires") else 1e-2
    return wl["t0"], wl["t1"], wl["save_t"], wl["atol"], atol_ratio


class Server:
    def __init__(self, slots: int = 4, budget_bytes: int = 64 << 30, max_pack: int = 1 << 21,
                 precision: str = "fp64", device: str = "cuda"):
        self.slots = slots
        self.budget = budget_bytes
        self.max_pack = max_pack
        self.precision = precision
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.clock0 = time.perf_counter()
        self._cv = threading.Condition()
        self._queue: collections.deque[Request] = collections.deque()
        self._inflight_bytes = 0
        self._free = list(range(slots))
        self._closed = False
        self._batches = 0
        self.batch_log = []
        self._ctx = [api.Context() for _ in range(slots)]
        self._streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self._work = [None] * slots
        self._slot_cv = [threading.Condition(self._cv) for _ in range(slots)]
        self._workers = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(slots)]
        self._sched = threading.Thread(target=self._scheduler, daemon=True)
        for t in self._workers:
            t.start()
        self._sched.start()

    def now(self) -> float:
        return time.perf_counter() - self.clock0

    def submit(self, req: Request) -> Request:
        with self._cv:
            if self._closed:
                raise RuntimeError("server closed")
            self._queue.append(req)
            self._cv.notify_all()
        return req

    def close(self):
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        self._sched.join()
        for t in self._workers:
            t.join()
        for c in self._ctx:
            c.close()

    # ---- scheduling -----------------------------------------------------
    def _take_batch(self):
        """Oldest request plus queued ones with its key (FIFO within the key)."""
        head = self._queue[0]
        batch, total = [], 0
        for r in list(self._queue):
            if r.key != head.key:
                continue
            if batch and total + r.n > self.max_pack:
                continue
            batch.append(r)
            total += r.n
        return batch, total

    def _scheduler(self):
        with self._cv:
            while True:
                while not self._closed and not (self._queue and self._free):
                    self._cv.wait()
                if self._closed and not self._queue:
                    if len(self._free) < self.slots:  # let the batches in flight finish first
                        self._cv.wait()
                        continue
                    for i in range(self.slots):
                        self._work[i] = "stop"
                        self._slot_cv[i].notify()
                    return
                if not self._free:
                    continue
                batch, total = self._take_batch()
                fp = record_footprint(batch[0].problem, total, batch[0].rtol)
                if self._inflight_bytes > 0 and self._inflight_bytes + fp > self.budget:
                    self._cv.wait()  # wait for memory to free up (head of line)
                    continue
                for r in batch:
                    self._queue.remove(r)
                slot = self._free.pop(0)
                self._inflight_bytes += fp
                self._work[slot] = (batch, fp, self._batches)
                self._batches += 1
                self._slot_cv[slot].notify()

    def _worker(self, i: int):
        torch.cuda.set_device(self.device)
        ctx, stream = self._ctx[i], self._streams[i]
        while True:
            with self._cv:
                while self._work[i] is None:
                    self._slot_cv[i].wait()
                job = self._work[i]
                self._work[i] = None
            if job == "stop":
                return
            batch, fp, bid = job
            t_start = self.now()
            try:
                self._run_batch(batch, ctx, stream)
            finally:
                t_done = self.now()
                for r in batch:
                    r.t_start, r.t_done, r.batch = t_start, t_done, bid
                    r.done.set()
                with self._cv:
                    self.batch_log.append((bid, i, len(batch), sum(r.n for r in batch), t_start, t_done))
                    self._inflight_bytes -= fp
                    self._free.append(i)
                    self._cv.notify_all()

    def _run_batch(self, batch, ctx, stream):
        problem, rtol = batch[0].key
        t0, t1, save_t, atol_fixed, ratio = _spec(problem)
        atol = rtol * ratio if ratio is not None else atol_fixed
        params = np.concatenate([r.params for r in batch])
        y0 = np.concatenate([r.y0 for r in batch])
        with torch.cuda.stream(stream):
            P = torch.from_numpy(np.ascontiguousarray(params.T)).pin_memory().to(self.device, non_blocking=True)
            Y = torch.from_numpy(np.ascontiguousarray(y0.T)).pin_memory().to(self.device, non_blocking=True)
            res = ctx.solve_grad(problem, P, Y, t0, t1, save_t, rtol, atol, layout="soa", check=False,
                                 precision=self.precision)
            loss = res["loss"].cpu().numpy()
            pb = res["params_bar"].cpu().numpy()
            yb = res["y0_bar"].cpu().numpy()
            st = res["status"].cpu().numpy()
        o = 0
        for r in batch:
            s = slice(o, o + r.n)
            r.loss, r.params_bar, r.y0_bar, r.status = loss[s], pb[:, s].T.copy(), yb[:, s].T.copy(), st[s]
            o += r.n


def c4_stream(num: int, seed: int = 0, log2n=(6, 20), problems=("lorenz", "vdp", "robertson"),
              rtols=(1e-6, 1e-8)):
    """The serving workload: each request draws its problem uniformly from
    `problems`, its ensemble size log-uniform in [2^log2n[0], 2^log2n[1]] and its
    rtol uniformly from `rtols`; inputs from the per-problem seeded ensembles."""
    u = W.uniform((seed << 8) ^ 0xC4, 3 * num)
    reqs = []
    for i in range(num):
        prob = problems[min(int(u[3 * i] * len(problems)), len(problems) - 1)]
        n = int(2.0 ** (log2n[0] + (log2n[1] - log2n[0]) * u[3 * i + 1]))
        rtol = rtols[min(int(u[3 * i + 2] * len(rtols)), len(rtols) - 1)]
        wl = W.make(prob, n, rtol=rtol, seed=1000 + i)
        reqs.append(Request(i, prob, wl["params"], wl["y0"], rtol))
    return reqs


def run_stream(server: Server, reqs, rate: float | None, seed: int = 0):
    """Submits reqs with Poisson arrivals at `rate` requests/s (None: all at once)
    and waits for all. Returns the requests (with timing filled in)."""
    gaps = np.zeros(len(reqs)) if rate is None else -np.log(1.0 - W.uniform(seed ^ 0xA77, len(reqs))) / rate
    start = server.now()
    t = start
    for r, g in zip(reqs, gaps):
        t += g
        delay = t - server.now()
        if delay > 0:
            time.sleep(delay)
        r.arrival = server.now()
        r.done.clear()
        server.submit(r)
    for r in reqs:
        r.done.wait()
    return reqs


def run_serial(reqs, precision="fp64", rate: float | None = None, seed: int = 0):
    """Baseline: plain launches, one request at a time in arrival order (no packing,
    no overlap). Returns per-request latencies with the same arrival process."""
    gaps = np.zeros(len(reqs)) if rate is None else -np.log(1.0 - W.uniform(seed ^ 0xA77, len(reqs))) / rate
    arrivals = np.cumsum(gaps)
    clock0 = time.perf_counter()
    lat = []
    for r, a in zip(reqs, arrivals):
        now = time.perf_counter() - clock0
        if now < a:
            time.sleep(a - now)
        t0, t1, save_t, atol_fixed, ratio = _spec(r.problem)
        atol = r.rtol * ratio if ratio is not None else atol_fixed
        P = torch.from_numpy(np.ascontiguousarray(r.params.T)).pin_memory().cuda(non_blocking=True)
        Y = torch.from_numpy(np.ascontiguousarray(r.y0.T)).pin_memory().cuda(non_blocking=True)
        res = api.solve_grad(r.problem, P, Y, t0, t1, save_t, r.rtol, atol, layout="soa", check=False,
                             precision=precision)
        for k in ("loss", "params_bar", "y0_bar", "status"):
            res[k].cpu()
        lat.append(time.perf_counter() - clock0 - a)
    return np.array(lat), time.perf_counter() - clock0


def latency_stats(lat):
    lat = np.asarray(lat)
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3)}
