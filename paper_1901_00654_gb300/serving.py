"""Continuous-batching request loop over the C ABI.

Requests (one smoothing problem each) arrive over time.  A dispatcher admits
a waiting request as soon as a slot is free and its estimated device memory
fits in the budget; each slot is a worker thread with its own CUDA stream, so
the kernels of all admitted requests overlap on the GPU.  Every request keeps
its sorted points and multigrid hierarchy resident in a plan from the moment
it is admitted until its coefficients are back on the host; plans are pooled
by grid shape, so a finished request's device memory is reused by the next
request of the same shape instead of being freed and allocated again.

All numerical work is done by libsps.so; this module only schedules.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import binding as B


def estimate_bytes(P: int, intervals, levels: int, n: int, itemsize: int = 8,
                   precision: int = B.SPS_PREC_MIXED) -> int:
    """Upper bound of the device memory of one plan after sps_set_points:
      * points: sorted coordinates (input type and an FP32 copy), responses,
        keys and permutation with their sort scratch, run lists per level;
      * about 30 coefficient vectors per level (FP64 and FP32 copies, the
        penalty and transfer temporaries, the PCG vectors);
      * the dense coarse solver: A_1, its inverse Cholesky factor and its
        transpose, and the scaled working copy (4 K_1^2 doubles);
      * the assembled stencils of the levels strictly between the coarsest
        and the finest, (2q+1)^P entries per coefficient where that fits the
        library's 8 GB per level (FP64; mixed plans hold an FP64 and an FP32
        copy while assembling);
      * FP64 plans: the precomputed basis values (and, for P = 3, products)
        of every point on every level above the coarsest."""
    Ks = []
    for g in range(levels):
        k = 1
        for N in intervals:
            k *= (N >> g) + 3
        Ks.append(k)                        # Ks[0] is the finest level
    K1 = Ks[-1]
    S = 7 ** P
    points = n * (P * itemsize + P * 4 + 8 + 16 + 8 + 12 * levels)
    vectors = sum(Ks) * 8 * 30
    coarse = K1 * K1 * 8 * 4
    stencil_bytes = 12 if precision == B.SPS_PREC_MIXED else 8
    stencils = sum(S * k * stencil_bytes for k in Ks[1:-1] if S * k * 8 <= 8e9)
    pre = 0
    if precision == B.SPS_PREC_FP64:
        pre = (levels - 1) * n * (4 * P + (20 if P == 3 else 0)) * 8
    return int(points + vectors + coarse + stencils + pre + (64 << 20))


@dataclass
class Completed:
    index: int
    t_arrival: float
    t_admit: float
    t_done: float
    coef: np.ndarray
    result: B.sps_result
    status: int

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


@dataclass
class ServerStats:
    completed: list = field(default_factory=list)
    makespan: float = 0.0
    peak_bytes: int = 0
    max_in_flight: int = 0

    def summary(self) -> dict:
        lat = np.array([c.latency for c in self.completed]) if self.completed else np.zeros(1)
        ok = sum(1 for c in self.completed if c.status == B.SPS_OK)
        return {"requests": len(self.completed), "converged": ok,
                "solves_per_s": len(self.completed) / self.makespan if self.makespan > 0 else 0.0,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "makespan_s": self.makespan, "peak_bytes": self.peak_bytes, "max_in_flight": self.max_in_flight}


class Server:
    """slots: concurrent requests on the GPU; budget_bytes: admission limit.

    executor / stream_factory replace the library call and the CUDA streams
    (both or neither): executor(problem, stream) -> (coef, sps_result, status)
    runs one request on the given stream.  The default runs it through
    libsps.so on torch CUDA streams; the replacements let the scheduler be
    exercised on its own."""

    def __init__(self, slots: int = 8, budget_bytes: float = 120e9, precision: int = B.SPS_PREC_MIXED,
                 tol: float = 1e-8, max_iter: int = 20000, pool_per_shape: int = 2, executor=None,
                 stream_factory=None):
        if (executor is None) != (stream_factory is None):
            raise ValueError("executor and stream_factory go together")
        self._executor = executor
        if stream_factory is None:
            import torch
            self.torch = torch
            stream_factory = torch.cuda.Stream
        self.slots = slots
        self.budget = int(budget_bytes)
        self.precision = precision
        self.tol = tol
        self.max_iter = max_iter
        self.pool_per_shape = pool_per_shape
        self._pool = collections.defaultdict(list)      # shape -> idle plans
        self._lock = threading.Lock()
        self._cv = threading.Condition(self._lock)
        self._used = 0
        self._in_flight = 0
        self._free_streams = [stream_factory() for _ in range(slots)]

    # ---------------------------------------------------------------- plans
    def _get_plan(self, pr):
        key = (pr.P, tuple(pr.intervals), pr.levels, tuple(pr.lo), tuple(pr.hi))
        with self._lock:
            lst = self._pool.get(key)
            pl = lst.pop() if lst else None
        if pl is None:
            pl = B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, precision=self.precision,
                        max_iter=self.max_iter)
        B.sps_set_lambda(pl.h, pr.lam)
        return key, pl

    def _put_plan(self, key, pl):
        with self._lock:
            if len(self._pool[key]) < self.pool_per_shape:
                self._pool[key].append(pl)
                return
        pl.close()

    def close(self):
        with self._lock:
            plans = [p for lst in self._pool.values() for p in lst]
            self._pool.clear()
        for p in plans:
            p.close()

    # ---------------------------------------------------------------- one request
    def _serve(self, idx, req, t0, est, stats):
        with self._lock:
            stream = self._free_streams.pop()
        t_admit = time.perf_counter() - t0
        if self._executor is not None:
            try:
                coef, res, status = self._executor(req.problem, stream)
            except Exception:   # a failed request must still release its slot and budget
                coef, res, status = None, B.sps_result(), B.SPS_EINTERNAL
            self._finish(idx, req, t_admit, t0, est, stats, stream, coef, res, status)
            return
        torch = self.torch
        try:
            with torch.cuda.stream(stream):
                key, pl = self._get_plan(req.problem)
                # device copies through torch's stream-ordered allocator: no cudaFree, so
                # the slots' streams never synchronise the whole device
                xd = torch.from_numpy(np.ascontiguousarray(req.problem.x)).to("cuda", non_blocking=True)
                yd = torch.from_numpy(np.ascontiguousarray(req.problem.y)).to("cuda", non_blocking=True)
                pl.set_points(xd, yd, stream=stream.cuda_stream)
                coef = np.zeros(pl.K)
                coef, res = pl.solve(self.tol, coef, stream=stream.cuda_stream, check=False)
                self._put_plan(key, pl)
            status = res.status
        except B.SpsError as e:
            coef, res, status = None, B.sps_result(), e.code
        except Exception:       # a failed request must still release its slot and budget
            coef, res, status = None, B.sps_result(), B.SPS_EINTERNAL
        self._finish(idx, req, t_admit, t0, est, stats, stream, coef, res, status)

    def _finish(self, idx, req, t_admit, t0, est, stats, stream, coef, res, status):
        t_done = time.perf_counter() - t0
        with self._cv:
            stats.completed.append(Completed(idx, req.t_arrival, t_admit, t_done, coef, res, status))
            self._used -= est
            self._in_flight -= 1
            self._free_streams.append(stream)
            self._cv.notify_all()

    # ---------------------------------------------------------------- the loop
    def run(self, trace, time_scale: float = 1.0) -> ServerStats:
        """Replay `trace` (workloads.Request list, sorted by arrival) in real
        time (arrival times multiplied by time_scale); returns per-request
        latencies and throughput."""
        stats = ServerStats()
        waiting = collections.deque()
        threads = []
        t0 = time.perf_counter()
        nxt = 0
        total = len(trace)
        while True:
            now = time.perf_counter() - t0
            while nxt < total and trace[nxt].t_arrival * time_scale <= now:
                waiting.append(nxt)
                nxt += 1
            with self._cv:
                while waiting:
                    i = waiting[0]
                    pr = trace[i].problem
                    est = estimate_bytes(pr.P, pr.intervals, pr.levels, pr.n, pr.x.dtype.itemsize,
                                         self.precision)
                    if self._in_flight >= self.slots or (self._used + est > self.budget and self._in_flight > 0):
                        break
                    waiting.popleft()
                    self._used += est
                    self._in_flight += 1
                    stats.peak_bytes = max(stats.peak_bytes, self._used)
                    stats.max_in_flight = max(stats.max_in_flight, self._in_flight)
                    req = trace[i]
                    req_scaled = type(req)(req.t_arrival * time_scale, req.problem)
                    th = threading.Thread(target=self._serve, args=(i, req_scaled, t0, est, stats), daemon=True)
                    th.start()
                    threads.append(th)
                done = len(stats.completed) == total
                if done:
                    break
                if nxt < total and not waiting:
                    timeout = max(0.0, trace[nxt].t_arrival * time_scale - (time.perf_counter() - t0))
                else:
                    timeout = 0.05
                self._cv.wait(timeout=min(timeout, 0.05))
        for th in threads:
            th.join()
        stats.makespan = time.perf_counter() - t0
        stats.completed.sort(key=lambda c: c.index)
        return stats
