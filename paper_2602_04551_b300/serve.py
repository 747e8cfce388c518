"""Serving loop: independent l0-l2 solves arriving over time, solved concurrently.

Each admitted request owns one handle (its X, G^-1 and node pool stay resident on
the device) and one CUDA stream.  The loop
  1. enqueues `rounds_per_step` branch-and-bound rounds on every admitted solve
     (asynchronous graph launches on their own streams, so the node batches of
     different solves overlap on the GPU);
  2. while those rounds run, admits arrived requests in arrival order while their
     device footprint (bnb_footprint) fits in the HBM budget (a request's data are
     generated and its per-tree setup is enqueued at admission);
  3. polls every solve; finished ones release their memory and record the
     time from arrival to a certified gap, split into the wait for admission
     (queueing) and the time from admission to the end (service).
The device work is all in the library's kernels; this module only schedules.
The backend is injectable so the scheduling logic is testable without a GPU.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Any, Callable

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    X: Any                          # (n, p) design, or None with `loader`
    y: Any
    lambda0: float
    lambda2: float
    M: float
    gap: float = 1e-4
    arrival: float = 0.0            # seconds after the start of the run
    options: dict = dataclasses.field(default_factory=dict)
    shape: tuple = None             # (n, p); taken from X when not given
    loader: Callable = None         # () -> (X, y, lambda0, M), called at admission

    def dims(self):
        return self.shape if self.shape is not None else self.X.shape

    def data(self):
        """(X, y, lambda0, M), generating them on first use when a loader is set."""
        if self.X is None:
            self.X, self.y, self.lambda0, self.M = self.loader()
        return self.X, self.y, self.lambda0, self.M


@dataclasses.dataclass
class Result:
    rid: int
    status: str
    ub: float
    lb: float
    nodes: int
    beta: np.ndarray
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def queueing(self) -> float:
        return self.admitted - self.arrival

    @property
    def service(self) -> float:
        return self.finished - self.admitted


class LibraryBackend:
    """The C-ABI library (one handle and one stream per solve)."""

    def __init__(self, device: int = 0):
        import paper_2602_04551_b300 as bnb
        self.bnb = bnb
        self.device = device

    def _options(self, req: Request, M=1.0):
        kw = dict(batch_K=256, queue_capacity=1 << 18, warm_capacity=1 << 14, device=self.device)
        kw.update(req.options)
        return self.bnb.bnb_options_default(M=M, **kw)

    def footprint(self, req: Request) -> int:
        n, p = req.dims()
        return self.bnb.bnb_footprint(n, p, self._options(req))

    def start(self, req: Request) -> Any:
        X, y, lam0, M = req.data()
        h = self.bnb.bnb_create(X, y, lam0, req.lambda2, self._options(req, M))
        self.bnb.bnb_solve_start(h, req.gap)
        if req.loader is not None:      # the handle holds its own copy on the device
            req.X = req.y = None
        return h

    def launch(self, h, rounds: int):
        self.bnb.bnb_solve_launch(h, rounds)

    def poll(self, h) -> dict:
        return self.bnb.bnb_solve_poll(h)

    def finish(self, h) -> dict:
        res = self.bnb.bnb_solve_finish(h)
        h.close()
        return res


class Server:
    def __init__(self, backend=None, budget_bytes: int = 150 << 30, rounds_per_step: int = 4,
                 clock: Callable[[], float] = time.perf_counter, sleep=time.sleep,
                 progress: Callable[[float, int, int, int], None] = None):
        self.backend = backend if backend is not None else LibraryBackend()
        self.budget = int(budget_bytes)
        self.rounds = int(rounds_per_step)
        self.clock = clock
        self.sleep = sleep
        self.peak_used = 0
        self.peak_active = 0
        self.admission_log = []       # (time, rid, footprint, used_after)
        self.progress = progress      # called once per loop pass: (time, pending, active, done)

    def run(self, requests: list[Request]) -> list[Result]:
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        active = {}                   # rid -> (req, handle, footprint, admitted_at)
        results = []
        used = 0
        t0 = self.clock()
        for r in pending:
            if self.backend.footprint(r) > self.budget:
                raise ValueError(f"request {r.rid} alone exceeds the HBM budget")
        while pending or active:
            # rounds first, so that admission work on the host overlaps them on the GPU
            for r, h, fp, _ in active.values():
                self.backend.launch(h, self.rounds)
            now = self.clock() - t0
            # admission: arrival order, while the footprint fits
            while pending and pending[0].arrival <= now:
                r = pending[0]
                fp = self.backend.footprint(r)
                if used + fp > self.budget:
                    break
                pending.pop(0)
                h = self.backend.start(r)
                used += fp
                active[r.rid] = (r, h, fp, self.clock() - t0)
                self.admission_log.append((self.clock() - t0, r.rid, fp, used))
            self.peak_used = max(self.peak_used, used)
            self.peak_active = max(self.peak_active, len(active))
            if not active:
                if pending:
                    self.sleep(max(0.0, pending[0].arrival - (self.clock() - t0)))
                continue
            done = []
            for rid, (r, h, fp, adm) in active.items():
                pr = self.backend.poll(h)
                if pr["done"]:
                    res = self.backend.finish(h)
                    results.append(Result(rid=rid, status=res["status"], ub=res["ub"], lb=res["lb"],
                                          nodes=res["nodes"], beta=res["beta"], arrival=r.arrival,
                                          admitted=adm, finished=self.clock() - t0))
                    done.append(rid)
                    used -= fp
            for rid in done:
                del active[rid]
            if self.progress is not None:
                self.progress(self.clock() - t0, len(pending), len(active), len(results))
        return sorted(results, key=lambda x: x.rid)


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times of a Poisson stream (exponential gaps of mean 1/rate)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def latency_summary(results: list[Result]) -> dict:
    """Latency from arrival to the end of each solve (p50/p99), split into queueing (arrival
    to admission) and service (admission to the end); solves/s over the whole stream; and
    how many solves ended certified (optimal or at the gap)."""
    lat = np.array([r.latency for r in results])
    que = np.array([r.queueing for r in results])
    ser = np.array([r.service for r in results])
    span = max(r.finished for r in results) - min(r.arrival for r in results)
    cert = [r for r in results if r.status in ("optimal", "gap")]
    pct = lambda a, q: float(np.percentile(a, q))
    return {"p50_s": pct(lat, 50), "p99_s": pct(lat, 99), "mean_s": float(lat.mean()),
            "queue_p50_s": pct(que, 50), "queue_p99_s": pct(que, 99),
            "service_p50_s": pct(ser, 50), "service_p99_s": pct(ser, 99),
            "solves_per_s": len(results) / span, "certified": len(cert),
            "certified_per_s": len(cert) / span,
            "makespan_s": span, "solves": len(results),
            "nodes": int(sum(r.nodes for r in results))}
