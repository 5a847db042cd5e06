"""Served form: a continuous-batching request loop over the asynchronous C ABI.

Requests (d, n_elem, p, ring radii, right-hand side) arrive over time.  A request is
admitted as soon as an in-flight slot is free and a problem handle of its shape is
ready; its solve is enqueued with ``iga_solve_async`` on that handle's stream and runs
on the device while later requests are admitted, so the work of many requests
overlaps.  Finished solves are detected by polling ``iga_solve_ready`` and retired
with ``iga_solve_collect``.

Problem handles are pooled by shape: a handle keeps its 1D factors, geometry
fields, Krylov workspace and captured CUDA graph resident, so a later request of the
same shape skips setup.  A shape seen for the first time is set up on a host worker
thread (eigen-factors, fields, workspace, graph capture) while the loop keeps
serving other requests; several shapes set up at once (their eigensolves run
concurrently on the device).  A waiting request whose shape already has an idle
handle is admitted ahead of older requests that still wait for a setup.  Admission of
new handles is bounded by a device-memory budget, and idle handles are evicted
least-recently-used when a new shape does not fit.  Every kernel reduces in a fixed
order, so a request's result does not depend on what else is in flight.
"""

import collections
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import torch

from .api import Problem

# bytes per DOF of a handle: fields, operator and FD scratch, vectors, and per Krylov
# vector V (FP64) plus Z (FP32 for TF32/BF16/TF32X3, FP64 otherwise); the error-compensated
# TF32 form holds its three FD scratch tensors twice (hi and lo parts)
_FIXED_PER_DOF = {2: 8 * (5 + 3 + 2 + 5) + 3 * 4, 3: 8 * (9 + 9 + 2 + 5) + 3 * 4}


def handle_bytes(d, N, max_iter, precision):
    z = 4 if precision in ("tf32", "bf16", "tf32x3") else (0 if precision == "none" else 8)
    # TF32X3: the FD scratch twice (hi and lo); FP64_TC: 8 BF16 slices and 2 FP64 intermediates
    split = 3 * 4 if precision == "tf32x3" else (8 * 2 + 2 * 8 if precision == "fp64tc" else 0)
    return int(N * (_FIXED_PER_DOF[d] + split + (max_iter + 1) * 8 + max_iter * z)) + (1 << 20)


class Request:
    __slots__ = ("rid", "t_arrival", "d", "n_elem", "p", "r0", "r1", "rhs", "key",
                 "t_admit", "t_done", "iters", "relres", "status", "x")

    def __init__(self, rid, t_arrival, d, n_elem, p, rhs, r0=1.0, r1=2.0):
        self.rid, self.t_arrival = rid, t_arrival
        self.d, self.n_elem, self.p, self.r0, self.r1 = d, n_elem, p, r0, r1
        self.rhs = rhs  # host float64 array, or a callable N -> array
        self.key = (d, n_elem, p, r0, r1)
        self.t_admit = self.t_done = None
        self.iters = self.relres = self.status = None
        self.x = None


class _Slot:
    def __init__(self, problem, nbytes, key):
        self.P = problem
        self.nbytes = nbytes
        self.key = key
        self.busy = False
        self.last_used = 0.0
        self.req = None
        self.b = torch.empty(problem.N, dtype=torch.float64, device=problem.device)
        self.x = torch.empty_like(self.b)
        self.h_rhs = torch.empty(problem.N, dtype=torch.float64, pin_memory=True)
        self.h_x = torch.empty(problem.N, dtype=torch.float64, pin_memory=True)


class Server:
    """Continuous batching of IGA solves on one GPU."""

    def __init__(self, precision="tf32", tol=1e-8, max_iter=100, max_inflight=32,
                 mem_budget=None, keep_solutions=False, device="cuda", setup_threads=4,
                 lookahead=4096, max_per_key=4, grid="throughput"):
        self.max_per_key = max_per_key
        self.grid = grid  # many solves run at once: few reduction blocks per solve
        self.precision, self.tol, self.max_iter = precision, tol, max_iter
        self.max_inflight = max_inflight
        self.device = torch.device(device)
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            mem_budget = int(0.7 * free)
        self.mem_budget = mem_budget
        self.keep_solutions = keep_solutions
        self.lookahead = lookahead
        self.pool = collections.defaultdict(list)  # key -> [slots]
        self.setting_up = {}  # key -> (future, bytes)
        self.reserved = 0
        self.setups = 0
        self.setup_s = 0.0
        self.setup_threads = setup_threads
        self.dropped = 0
        self.executor = ThreadPoolExecutor(max_workers=setup_threads)

    # ---------------------------------------------------------------- pool
    def _setup(self, key, nbytes):
        d, n_elem, p, r0, r1 = key
        t = time.perf_counter()
        with torch.cuda.device(self.device):
            P = Problem(d, n_elem, p, "annulus", r0, r1, precision=self.precision,
                        device=self.device, stream=torch.cuda.Stream(self.device),
                        grid=self.grid)
            P.prepare(1, self.max_iter)
            slot = _Slot(P, nbytes, key)
        return slot, time.perf_counter() - t

    def _evict_until(self, need):
        idle = sorted((s for ss in self.pool.values() for s in ss if not s.busy),
                      key=lambda s: s.last_used)
        for s in idle:
            if self.reserved + need <= self.mem_budget:
                break
            self.pool[s.key].remove(s)
            s.P.close()
            self.reserved -= s.nbytes
        return self.reserved + need <= self.mem_budget

    def _harvest_setups(self):
        for key, (fut, nbytes) in list(self.setting_up.items()):
            if fut.done():
                del self.setting_up[key]
                slot, dt = fut.result()
                self.setup_s += dt
                self.pool[key].append(slot)

    def _needs_setup(self, key):
        """True if a new handle of this shape should be set up now: none is being set up,
        every existing one is busy, and the per-shape limit allows another."""
        if key in self.setting_up:
            return False
        slots = self.pool.get(key, [])
        return len(slots) < self.max_per_key and all(s.busy for s in slots)

    def _start_setup(self, req):
        """Reserve memory (evicting idle handles least recently used first) and submit the
        setup of a handle of the request's shape; False if it does not fit now."""
        N = (req.n_elem + req.p - 2) ** req.d
        need = handle_bytes(req.d, N, self.max_iter, self.precision)
        if need > self.mem_budget:
            raise RuntimeError(f"request {req.rid} needs {need} bytes, above the budget")
        if not self._evict_until(need):
            return False
        self.reserved += need
        self.setups += 1
        self.setting_up[req.key] = (self.executor.submit(self._setup, req.key, need), need)
        return True

    # ---------------------------------------------------------------- request life
    def _start(self, s, req, now):
        s.busy, s.req = True, req
        s.last_used = now
        req.t_admit = now
        rhs = req.rhs(s.P.N) if callable(req.rhs) else req.rhs
        s.h_rhs.copy_(torch.from_numpy(np.ascontiguousarray(rhs, dtype=np.float64)))
        with torch.cuda.stream(s.P.stream):
            s.b.copy_(s.h_rhs, non_blocking=True)
        s.P.solve_async(s.b, s.x, tol=self.tol, max_iter=self.max_iter)
        with torch.cuda.stream(s.P.stream):
            s.h_x.copy_(s.x, non_blocking=True)

    def _finish(self, s, now):
        info = s.P.collect()
        s.P.stream.synchronize()  # the host copy of x queued after the solve
        req = s.req
        req.t_done = time.perf_counter()
        req.iters = int(info["iters"][0])
        req.relres = float(info["relres_true"][0])
        req.status = int(info["status"][0])
        if self.keep_solutions:
            req.x = s.h_x.numpy().copy()
        s.busy, s.req = False, None
        s.last_used = now

    # ---------------------------------------------------------------- loop
    def run(self, requests, realtime=True, time_limit=None):
        """Serve ``requests`` (t_arrival in seconds from the start).  With ``realtime``
        a request becomes visible at its arrival time; otherwise all are queued at
        once.  Admission: a waiting request whose shape has an idle handle starts at once
        (oldest first, up to ``max_inflight`` solves in flight); shapes without a free
        handle get one set up on the worker threads, oldest waiting request first, at
        most ``setup_threads`` setups at a time.  At ``time_limit`` no new request is
        admitted: waiting ones are dropped (counted in ``self.dropped``) and the solves in
        flight drain.  Returns the completed requests."""
        pending = collections.deque(sorted(requests, key=lambda r: r.t_arrival))
        waiting = {}                   # shape -> deque of requests, arrival order
        order = collections.deque()    # every waiting request, arrival order (lazily pruned)
        nwait = 0
        inflight = []
        done = []
        self.dropped = 0
        t0 = time.perf_counter()
        while pending or nwait or inflight or self.setting_up:
            now = time.perf_counter()
            rel = now - t0
            closed = time_limit is not None and rel > time_limit
            if closed and (pending or nwait):
                self.dropped += len(pending) + nwait
                pending.clear()
                waiting.clear()
                order.clear()
                nwait = 0
            while pending and (not realtime or pending[0].t_arrival <= rel):
                r = pending.popleft()
                r.t_arrival = t0 + (r.t_arrival if realtime else 0.0)
                waiting.setdefault(r.key, collections.deque()).append(r)
                order.append(r)
                nwait += 1
            still = []
            for s in inflight:
                if s.P.ready():
                    req = s.req
                    self._finish(s, now)
                    done.append(req)
                else:
                    still.append(s)
            inflight = still
            self._harvest_setups()
            # warm shapes: the oldest waiting request of every shape with an idle handle
            cands = []
            for key, dq in waiting.items():
                if dq and any(not s.busy for s in self.pool.get(key, [])):
                    cands.append((dq[0].t_arrival, dq[0].rid, key))
            cands.sort()
            for _, _, key in cands:
                for s in self.pool[key]:
                    if len(inflight) >= self.max_inflight or not waiting[key]:
                        break
                    if s.busy:
                        continue
                    req = waiting[key].popleft()
                    nwait -= 1
                    self._start(s, req, time.perf_counter())
                    inflight.append(s)
                if not waiting[key]:
                    del waiting[key]
            # cold shapes: set up handles for the oldest waiting requests that need one
            while order and order[0].t_admit is not None:
                order.popleft()
            if not closed and len(self.setting_up) < self.setup_threads:
                scanned = 0
                for r in order:
                    if len(self.setting_up) >= self.setup_threads or scanned >= self.lookahead:
                        break
                    scanned += 1
                    if r.t_admit is None and self._needs_setup(r.key):
                        if not self._start_setup(r):
                            break
            if not pending and not nwait and not inflight and not self.setting_up:
                break
            time.sleep(0)
        return done

    def close(self):
        self.executor.shutdown(wait=True)
        self._harvest_setups()
        for slots in self.pool.values():
            for s in slots:
                s.P.close()
        self.pool.clear()
        self.reserved = 0


def latency_stats(done):
    if len(done) == 0:
        return {"completed": 0}
    lat = np.array([(r.t_done - r.t_arrival) * 1e3 for r in done])
    span = max(r.t_done for r in done) - min(r.t_arrival for r in done)
    return {"completed": len(done), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "solves_per_s": len(done) / span if span > 0 else None,
            "dof_iters": float(sum((r.n_elem + r.p - 2) ** r.d * r.iters for r in done)),
            "span_s": span}
