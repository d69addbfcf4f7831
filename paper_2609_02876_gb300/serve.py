"""Continuous-batching request server for gradient requests (one GPU).

A request is one ensemble: (problem, params (n, P), y0 (n, d), rtol), host
arrays. The server keeps `slots` solve contexts (each its own device
workspace and CUDA stream, driven by one host thread). Work is queued as
items: a request of at most `max_chunk` trajectories is one item; a larger
one is cut into chunks of `max_chunk` trajectories, its items queued in a
second FIFO. Whenever a slot is free it takes, in this order:
  - the oldest small request, packed with every other queued small request of
    the same (problem, rtol) behind it, up to `max_pack` trajectories, into
    ONE launch of the persistent record + reverse kernels;
  - else the oldest chunk of a large request.
So small requests pass large ones at chunk boundaries, and the chunks of the
large requests run in arrival order, each request's chunks side by side on
the free slots. Trajectories are independent, so each request's results are
exactly those of solving it alone (tested). A launch is admitted only if the
estimated record footprint of all launches in flight stays within
`budget_bytes`; launches on different slots overlap on the device. Latency =
completion of a request's last item - arrival. `max_chunk=None` turns the
chunking off (every request one item, packed up to `max_pack`).

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
    left: int = 0  # items not yet completed
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


@dataclass(eq=False)
class Item:
    """Trajectories [lo, hi) of one request: the unit the scheduler packs."""
    req: Request
    lo: int
    hi: int

    @property
    def n(self) -> int:
        return self.hi - self.lo

    @property
    def key(self):
        return self.req.key


def pack_batch(queue, limit):
    """The oldest item of `queue` plus the queued items with its key behind it,
    in arrival order, while the total stays within `limit` (an item larger than
    the limit still runs, alone)."""
    head = queue[0]
    batch, total = [], 0
    for it in list(queue):
        if it.key != head.key:
            continue
        if batch and total + it.n > limit:
            continue
        batch.append(it)
        total += it.n
    return batch, total


def _spec(problem):
    """Time span, save times and atol rule of a problem's workload."""
    wl = W.make(problem, 1)
    atol_ratio = None if problem in ("robertson", "hires") else 1e-2
    return wl["t0"], wl["t1"], wl["save_t"], wl["atol"], atol_ratio


class Server:
    def __init__(self, slots: int = 4, budget_bytes: int = 64 << 30, max_pack: int = 1 << 21,
                 precision: str = "fp64", device: str = "cuda", max_chunk: int | None = None):
        self.slots = slots
        self.budget = budget_bytes
        self.max_chunk = max_chunk
        self.max_pack = max_pack if max_chunk is None else min(max_pack, max_chunk)
        self.precision = precision
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.clock0 = time.perf_counter()
        self._cv = threading.Condition()
        self._small: collections.deque[Item] = collections.deque()
        self._large: collections.deque[Item] = collections.deque()
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
        d, P = req.y0.shape[1], req.params.shape[1]
        req.loss = np.empty(req.n)
        req.params_bar = np.empty((req.n, P))
        req.y0_bar = np.empty((req.n, d))
        req.status = np.empty(req.n, np.int32)
        req.t_start = math.nan
        if self.max_chunk is not None and req.n > self.max_chunk:
            items = [Item(req, lo, min(lo + self.max_chunk, req.n)) for lo in range(0, req.n, self.max_chunk)]
            queue = self._large
        else:
            items, queue = [Item(req, 0, req.n)], self._small
        req.left = len(items)
        with self._cv:
            if self._closed:
                raise RuntimeError("server closed")
            queue.extend(items)
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
        """Small requests first (packed by key), else the oldest large-request chunk."""
        if self._small:
            return pack_batch(self._small, self.max_pack), self._small
        return ([self._large[0]], self._large[0].n), self._large

    def _scheduler(self):
        with self._cv:
            while True:
                queued = bool(self._small or self._large)
                while not self._closed and not (queued and self._free):
                    self._cv.wait()
                    queued = bool(self._small or self._large)
                if self._closed and not queued:
                    if len(self._free) < self.slots:  # let the launches in flight finish first
                        self._cv.wait()
                        continue
                    for i in range(self.slots):
                        self._work[i] = "stop"
                        self._slot_cv[i].notify()
                    return
                if not self._free:
                    continue
                (batch, total), queue = self._take_batch()
                fp = record_footprint(batch[0].req.problem, total, batch[0].req.rtol)
                if self._inflight_bytes > 0 and self._inflight_bytes + fp > self.budget:
                    self._cv.wait()  # wait for memory to free up (head of line)
                    continue
                for it in batch:
                    queue.remove(it)
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
                with self._cv:
                    for it in batch:
                        r = it.req
                        if not r.t_start <= t_start:
                            r.t_start = t_start
                        r.batch = bid
                        r.left -= 1
                        if r.left == 0:
                            r.t_done = t_done
                            r.done.set()
                    self.batch_log.append((bid, i, len(batch), sum(it.n for it in batch), t_start, t_done))
                    self._inflight_bytes -= fp
                    self._free.append(i)
                    self._cv.notify_all()

    def _run_batch(self, batch, ctx, stream):
        problem, rtol = batch[0].key
        t0, t1, save_t, atol_fixed, ratio = _spec(problem)
        atol = rtol * ratio if ratio is not None else atol_fixed
        params = np.concatenate([it.req.params[it.lo:it.hi] for it in batch])
        y0 = np.concatenate([it.req.y0[it.lo:it.hi] for it in batch])
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
        for it in batch:
            s, r = slice(o, o + it.n), it.req
            r.loss[it.lo:it.hi] = loss[s]
            r.params_bar[it.lo:it.hi] = pb[:, s].T
            r.y0_bar[it.lo:it.hi] = yb[:, s].T
            r.status[it.lo:it.hi] = st[s]
            o += it.n


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
