"""Continuous-batching serving loop for Helmholtz solves (host scheduler over the C ABI).

Requests (grid n, medium, point source) arrive over time. Each is served by a *resident*
problem: the hierarchy for its medium is built once and kept on the device, so later requests
with the same medium only bring a new right-hand side. Admission is by device memory: a request
starts only when its problem is resident and idle, or when a new problem's footprint
(``hz_footprint_bytes`` plus its right-hand side and solution) fits the budget, evicting idle
problems of other media if needed. Admitted solves run through the non-blocking entry points
(``hz_solve_start`` / ``hz_solve_poll`` / ``hz_solve_finish``): each problem has its own stream,
so solves of different requests overlap on the GPU while the loop keeps polling, admitting new
requests as soon as slots and memory free up. Each request's result depends only on its own
inputs (no shared state, deterministic reductions), so it is bitwise the same alone and in the
mix.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Job:
    rid: int
    n: int
    key: tuple  # medium key: requests with equal keys share a resident hierarchy
    kfield_fn: object  # () -> (n+1, n+1) float64 k field (called when the hierarchy is built)
    k_ref: float
    source: tuple  # (i, j) node of the point source, value 1/h^2
    arrival: float = 0.0
    start: float | None = None
    end: float | None = None
    result: dict = field(default_factory=dict)
    precision: str | None = None  # None: the server's; set to "fp64" when a solve falls back


def device_io(n: int, source: tuple):
    """Right-hand side (point source 1/h^2 at `source`) and solution buffers on the device."""
    import torch

    rhs = torch.zeros((n + 1, n + 1), dtype=torch.complex128, device="cuda")
    i, j = source
    rhs[j, i] = float(n * n)
    return rhs, torch.empty_like(rhs)


class Server:
    """The serving loop. ``keep_solutions``: True copies every solution to the host (in the job's
    result), a set of request ids only those requests' solutions. ``fallback``: a request whose
    FP32-form solve ends without reaching the tolerance (maxit or breakdown: FP32 rounding of the
    V-cycle can stall a long Bi-CGSTAB run that the FP64 form completes) is solved again at once by
    the FP64 form; its result records the first attempt."""

    ENOMEM = 2  # hz_status of a request whose hierarchy can never fit the budget

    def __init__(self, hbm_budget: int, precision: str = "fp32", tol: float = 1e-6, maxit: int = 4000,
                 max_active: int = 32, variant: str = "hyb", keep_solutions=False, backend=None,
                 make_io=device_io, fallback: bool = True):
        if backend is None:
            from . import hz as backend
        self.hz = backend
        self.make_io = make_io
        self.budget = int(hbm_budget)
        self.precision = precision
        self.tol = tol
        self.maxit = maxit
        self.max_active = max_active
        self.variant = variant
        self.keep = keep_solutions
        self.fallback = fallback
        self.fallbacks = 0
        self.queue = collections.deque()
        self.active = []  # (job, problem, rhs, x)
        self.idle = collections.OrderedDict()  # key -> list of idle problems (LRU order)
        self.used = 0
        self.done = []
        self.peak_used = 0
        self.peak_active = 0
        self.evictions = 0

    # ------------------------------------------------------------------ memory
    def footprint(self, n: int, precision: str | None = None) -> int:
        prec = precision or self.precision
        return self.hz.footprint_bytes(n, precision=prec, variant=self.variant) + 2 * 16 * (n + 1) ** 2

    def _prec(self, job: Job) -> str:
        return job.precision or self.precision

    def _key(self, job: Job) -> tuple:
        return (job.key, self._prec(job))

    def _evict_for(self, need: int) -> bool:
        while self.used + need > self.budget and self.idle:
            key, plist = next(iter(self.idle.items()))
            prob = plist.pop()
            if not plist:
                del self.idle[key]
            self.used -= self.footprint(prob.n, prob.key[1])
            prob.close()
            self.evictions += 1
        return self.used + need <= self.budget

    def _acquire(self, job: Job):
        key = self._key(job)
        plist = self.idle.get(key)
        if plist:
            prob = plist.pop()
            if not plist:
                del self.idle[key]
            return prob
        need = self.footprint(job.n, self._prec(job))
        if not self._evict_for(need):
            return None
        prob = self.hz.Problem(job.n, job.kfield_fn(), 0.5, variant=self.variant, precision=self._prec(job),
                               k_ref=job.k_ref)
        prob.key = key
        self.used += need
        self.peak_used = max(self.peak_used, self.used)
        return prob

    def _release(self, prob):
        self.idle.setdefault(prob.key, []).append(prob)
        self.idle.move_to_end(prob.key)

    # ------------------------------------------------------------------ loop
    def submit(self, job: Job):
        self.queue.append(job)

    def _reject(self, job: Job, now: float, status: int, why: str):
        job.start = job.end = now
        job.result = {"status": status, "error": why, "iterations": 0.0}
        self.done.append(job)

    def _admit(self, now: float):
        while self.queue and len(self.active) < self.max_active:
            job = self.queue[0]
            if self._key(job) not in self.idle and self.footprint(job.n, self._prec(job)) > self.budget:
                # no amount of eviction makes room: fail the request instead of waiting forever
                self.queue.popleft()
                self._reject(job, now, self.ENOMEM, "footprint exceeds the device-memory budget")
                continue
            prob = self._acquire(job)
            if prob is None:
                break  # memory full: wait for a solve to finish
            self.queue.popleft()
            rhs, x = self.make_io(job.n, job.source)
            job.start = now
            prob.solve_start(rhs, x, tol=self.tol, maxit=self.maxit)
            self.active.append((job, prob, rhs, x))
            self.peak_active = max(self.peak_active, len(self.active))

    def _poll(self, now_fn):
        still = []
        for job, prob, rhs, x in self.active:
            if prob.solve_poll():
                x, info, _ = prob.solve_finish(history_cap=0, allow_fail=True)
                if info["status"] != 0 and self.fallback and self._prec(job) == "fp32":
                    # solve it again with the FP64 V-cycle, ahead of the queue
                    job.result = {"fp32_attempt": dict(info)}
                    job.precision = "fp64"
                    self.fallbacks += 1
                    self._release(prob)
                    self.queue.appendleft(job)
                    continue
                job.end = now_fn()
                first = job.result.get("fp32_attempt")
                job.result = dict(info)
                if first is not None:
                    job.result["fp32_attempt"] = first
                if self.keep is True or (self.keep and job.rid in self.keep):
                    job.result["x"] = x.cpu().numpy()
                self.done.append(job)
                self._release(prob)
            else:
                still.append((job, prob, rhs, x))
        self.active = still

    def run(self, jobs, realtime: bool = True, time_limit: float | None = None):
        """Serve `jobs` (sorted by arrival, seconds from start). Returns a summary dict."""
        pending = collections.deque(sorted(jobs, key=lambda j: j.arrival))
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        while pending or self.queue or self.active:
            t = now()
            if time_limit is not None and t > time_limit:
                break
            while pending and (not realtime or pending[0].arrival <= t):
                self.submit(pending.popleft())
            self._admit(t)
            self._poll(now)
            if not self.active and not self.queue and pending and realtime:
                time.sleep(max(0.0, min(0.002, pending[0].arrival - now())))
        wall = now()
        return self.summary(wall)

    def summary(self, wall: float) -> dict:
        ok = [j for j in self.done if j.result.get("status") == 0]
        lat = np.array([(j.end - j.arrival) * 1e3 for j in self.done]) if self.done else np.zeros(0)
        return {
            "completed": len(self.done),
            "converged": len(ok),
            "wall_s": wall,
            "solves_per_s": len(self.done) / wall if wall > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "peak_hbm_bytes": self.peak_used,
            "peak_active": self.peak_active,
            "evictions": self.evictions,
            "fp64_fallbacks": self.fallbacks,
            "statuses": dict(collections.Counter(int(j.result.get("status", -1)) for j in self.done)),
        }

    def close(self):
        for _, prob, _, _ in self.active:
            try:
                prob.solve_finish(history_cap=0, allow_fail=True)
            except Exception:
                pass
            prob.close()
        for plist in self.idle.values():
            for prob in plist:
                prob.close()
        self.active, self.idle = [], collections.OrderedDict()
