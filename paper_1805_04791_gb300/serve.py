"""Continuous-batching serving loop for scattering solves.

Requests (kind, grid size, frequency, medium seed, incident wave) arrive over
time.  The server admits a waiting request as soon as its device-memory need
(from ``vie_problem_bytes``) fits the HBM budget and a slot is free; every
admitted request runs in its own worker thread on its own CUDA stream: medium
set-up, kernel transforms, right-hand side and the mixed-precision GMRES solve.
The library allocates stream-ordered and holds no device-wide locks, so the
kernels of all admitted requests overlap on the GPU; when a request finishes,
its memory returns to the budget and the next waiting request is admitted.

Admission order is shortest job first (work estimated as n^3), with aging: a
request that has waited ``max_wait_s`` is admitted ahead of smaller ones, so
large grids are not starved.  Before the first arrival the server chooses the
z-pass schedule of every grid size it may see (``pretune``) on an otherwise
idle GPU: a choice timed while other requests load the device would be
distorted, and the choice is kept for the whole process.

Each result records arrival, admission, completion, residual and the solution
norm; latency percentiles and throughput summarise a run.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import (VIE_HELMHOLTZ, VIE_MAXWELL, VIE_SOLVE_MIXED, Problem, vie_problem_bytes)


@dataclass
class ServeResult:
    rid: int
    kind: str
    n: int
    arrival_s: float
    admit_s: float = 0.0
    done_s: float = 0.0
    rel_residual: float = float("nan")
    status: str = "pending"
    gmres_iters: int = 0
    solution_norm: float = float("nan")
    solution: object = None

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


@dataclass
class ServeStats:
    results: list = field(default_factory=list)
    wall_s: float = 0.0
    peak_bytes: int = 0
    peak_slots: int = 0

    def summary(self) -> dict:
        lat = sorted(r.latency_s for r in self.results if r.status == "ok")
        ok = len(lat)

        def q(p):
            return lat[min(ok - 1, int(round(p / 100.0 * (ok - 1))))] if ok else None

        return {"requests": len(self.results), "completed": ok,
                "failed": sum(r.status != "ok" for r in self.results),
                "p50_latency_s": q(50), "p99_latency_s": q(99), "solves_per_s": ok / self.wall_s if self.wall_s else None,
                "wall_s": self.wall_s, "peak_inflight": self.peak_slots, "peak_bytes": self.peak_bytes}


class Server:
    """Admits requests by HBM budget and runs each on its own stream and thread."""

    def __init__(self, budget_bytes: float = 160e9, max_slots: int = 32, restart: int = 30, tol: float = 1e-8,
                 inner_tol: float = 1e-5, keep_solutions: bool = False, device: int = 0, policy: str = "sjf",
                 max_wait_s: float = 30.0):
        self.budget = int(budget_bytes)
        self.max_slots = max_slots
        self.restart = restart
        self.tol = tol
        self.inner_tol = inner_tol
        self.keep = keep_solutions
        self.device = device
        self.policy = policy
        self.max_wait_s = max_wait_s

    def pretune(self, sizes, kinds=("helmholtz",)):
        """Choose the FP32 z-pass schedule of every grid size in ``sizes`` now (one
        small problem per size, on this thread, GPU otherwise idle).  Helmholtz and
        Maxwell with mu = I use the same kernel set, hence the same choice."""
        import torch

        import vie_inputs as vi

        from . import VIE_FP32

        torch.cuda.set_device(self.device)
        dev = torch.device("cuda", self.device)
        for n in sorted(set(sizes)):
            for kind in kinds:
                eps = vi.bump_medium_torch(n, 1, dev)
                P = Problem(kind, n, -1.0, 1.0, 2.0 * np.pi, eps, None)
                try:
                    P.tune(VIE_FP32)
                finally:
                    P.close()
                del eps
        torch.cuda.synchronize()

    def request_bytes(self, req) -> int:
        kind = VIE_HELMHOLTZ if req.kind == "helmholtz" else VIE_MAXWELL
        n3 = req.n ** 3
        # handle (set-up peak or steady state) + eps + rhs + solution buffers
        return vie_problem_bytes(kind, req.n, 1, self.restart, 0) + 9 * n3 * 16 + 2 * 3 * n3 * 16

    def _solve(self, req, res: ServeResult, done_cb):
        import torch

        import vie_inputs as vi

        P = None
        try:
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                dev = torch.device("cuda", self.device)
                eps = vi.bump_medium_torch(req.n, req.seed, dev)
                omega = 2.0 * np.pi * req.wavelengths / 2.0
                P = Problem(req.kind, req.n, -1.0, 1.0, omega, eps, None, stream=stream)
                b = torch.empty((P.ncomp, req.n, req.n, req.n), dtype=torch.complex128, device=dev)
                pol = req.polarisation if req.kind == "maxwell" else None
                P.rhs(req.direction, pol, 1, b, stream=stream)
                J = torch.zeros_like(b)
                st, info = P.solve(b, J, tol=self.tol, restart=self.restart, max_outer=40, max_inner=4000,
                                   inner_tol=self.inner_tol, mode=VIE_SOLVE_MIXED, stream=stream, allow_noconv=True)
                stream.synchronize()
                res.rel_residual = info.rel_residual
                res.gmres_iters = info.inner_iters
                res.solution_norm = float(torch.linalg.vector_norm(J).item())
                if self.keep:
                    res.solution = J.cpu().numpy()
                res.status = "ok" if st == 0 else "noconv"
                del eps, b, J
        except Exception as e:  # a failed request frees its slot and is reported
            res.status = f"error: {e}"
        finally:
            # the handle's device memory goes back before the slot does (destroy
            # frees stream-ordered on the handle's stream and waits for it)
            if P is not None:
                try:
                    P.close()
                except Exception as e:
                    if res.status == "ok":
                        res.status = f"error: {e}"
            done_cb(res)

    def run(self, requests, time_scale: float = 1.0) -> ServeStats:
        """Replay ``requests`` (sorted by arrival_s, seconds) in real time; blocks until all finish."""
        pending = deque(sorted(requests, key=lambda r: r.arrival_s))
        queue = deque()
        cv = threading.Condition()
        state = {"used": 0, "slots": 0, "finished": 0}
        stats = ServeStats()
        sizes = {}
        t0 = time.perf_counter()
        total = len(pending)
        threads = []

        def done(res):
            with cv:
                res.done_s = time.perf_counter() - t0
                state["used"] -= sizes[res.rid]
                state["slots"] -= 1
                state["finished"] += 1
                cv.notify_all()

        with cv:
            while state["finished"] < total:
                now = time.perf_counter() - t0
                while pending and pending[0].arrival_s * time_scale <= now:
                    queue.append(pending.popleft())
                # admission by budget and slot count: shortest job first (n^3), except
                # that requests waiting longer than max_wait_s go first (oldest first)
                while queue:
                    if self.policy == "fifo":
                        req = queue[0]
                    else:
                        old = [q for q in queue if now - q.arrival_s * time_scale >= self.max_wait_s]
                        req = old[0] if old else min(queue, key=lambda q: (q.n, q.arrival_s))
                    need = sizes.setdefault(req.rid, self.request_bytes(req))
                    if need > self.budget:
                        queue.remove(req)
                        r = ServeResult(req.rid, req.kind, req.n, req.arrival_s * time_scale, now, now,
                                        status="rejected: exceeds budget")
                        stats.results.append(r)
                        state["finished"] += 1
                        continue
                    if state["slots"] >= self.max_slots or state["used"] + need > self.budget:
                        break
                    queue.remove(req)
                    state["used"] += need
                    state["slots"] += 1
                    stats.peak_bytes = max(stats.peak_bytes, state["used"])
                    stats.peak_slots = max(stats.peak_slots, state["slots"])
                    res = ServeResult(req.rid, req.kind, req.n, req.arrival_s * time_scale, now)
                    stats.results.append(res)
                    th = threading.Thread(target=self._solve, args=(req, res, done), daemon=True)
                    threads.append(th)
                    th.start()
                if state["finished"] >= total:
                    break
                wait = 0.05
                if pending:
                    wait = max(0.0, min(wait, pending[0].arrival_s * time_scale - (time.perf_counter() - t0)))
                cv.wait(timeout=wait if wait > 0 else 0.001)
        for th in threads:
            th.join()
        stats.wall_s = time.perf_counter() - t0
        stats.results.sort(key=lambda r: r.rid)
        return stats
