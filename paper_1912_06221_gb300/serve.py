"""Continuous-batching solve server on one GPU.

Requests (a mesh, order, element-wise D, velocity, initial state and a number of SSP-RK3
steps) arrive over time.  Every admitted request stays resident on the device in its own
library context and CUDA stream; the scheduler advances all resident requests in chunks of
steps (replayed CUDA graphs), keeping at most two chunks queued per request, so kernels of
different requests overlap on the GPU while the host keeps returning to admission.  Waiting
requests are admitted as slots and device memory free up: admission compares the context's
device bytes (rdg_query_bytes on an upper bound of the edge count, plus set-up scratch) with
the budget still free, and the set-up (mesh upload, FP64 operator build, step-size power
iteration, initial state) runs on a worker thread.  A finished request's state is copied
back and its context released at once.  Latency is completion time minus arrival time.
All device work is the library's; this module only schedules.
"""
from __future__ import annotations

import math
import threading
import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

from . import rdg


@dataclass
class SolveRequest:
    rid: int
    arrival: float                 # seconds from the start of the run
    xy: Optional[np.ndarray]       # None: built by `build` during set-up
    tri: Optional[np.ndarray]
    N: int
    D_elem: Optional[np.ndarray]
    v: tuple
    u0: Callable                   # u0(x, y) evaluated at the library's node coordinates
    steps: int
    dt: Optional[float] = None     # None: 0.5 x the stability bound (power iteration)
    precision: int = rdg.FP32
    # the paper's Algorithm 1: the requests' element-wise D jumps by up to 1e4 across an
    # interface, where Algorithm 2's operator has growing modes and Algorithm 1's does not
    interface: int = rdg.IFACE_ALG1
    build: Optional[Callable] = None   # () -> (xy, tri, D_elem), run on the set-up worker
    n_triangles: int = 0           # triangle count when the mesh is built lazily


@dataclass
class SolveResult:
    rid: int
    arrival: float
    admitted: float
    started: float
    finished: float
    K: int
    Np: int
    steps: int
    dt: float
    state: np.ndarray = field(repr=False)

    @property
    def latency(self):
        return self.finished - self.arrival

    @property
    def dof_updates(self):
        return self.K * self.Np * 3 * self.steps


SSP_RK3_REAL_EXTENT = 2.5127


def spectral_radius(solver, torch, iters=30, seed=0):
    """Power iteration on the library right-hand side, on the current stream, with a single
    host synchronisation at the end (the normalisation stays on the device, so the
    iterations do not wait behind other requests' queued work one by one)."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn((solver.K, solver.Np), generator=g, device="cuda", dtype=solver.dtype)
    y = torch.empty_like(x)
    for _ in range(iters):
        x /= torch.linalg.vector_norm(x)
        solver.rhs_eval(x, y, 0.0)
        x, y = y, x
    return float(torch.linalg.vector_norm(x))


def edge_count_bound(tri: np.ndarray) -> int:
    """Distinct vertex pairs of the triangles: an upper bound on the library's edge count
    (periodic identification can only merge further edges)."""
    t = np.asarray(tri, np.int64)
    a = np.concatenate([t[:, 0], t[:, 1], t[:, 2]])
    b = np.concatenate([t[:, 1], t[:, 2], t[:, 0]])
    key = np.minimum(a, b) * (int(t.max()) + 1) + np.maximum(a, b)
    return int(np.unique(key).size)


def request_bytes(req: SolveRequest) -> int:
    """Device bytes a request holds while resident, plus its set-up scratch."""
    if req.tri is not None:
        nt = int(req.tri.shape[0])
        E = edge_count_bound(req.tri)
    else:   # lazily built unit-square mesh: E <= 3K/2 plus the boundary
        nt = int(req.n_triangles)
        E = 3 * nt // 2 + 4 * int(math.sqrt(nt)) + 8
    resident = rdg.query_bytes(req.N, nt, E, E, req.precision, 0, 0)
    scratch = nt * 6 * 8 + nt * 8 + E * (16 + 16) + (1 << 20)   # FP64 set-up copies and tables
    power = 2 * nt * rdg.np_of(req.N) * (8 if req.precision == rdg.FP64 else 4)
    return resident + scratch + power


class _Active:
    def __init__(self, req, solver, stream, admitted, started, dt, nbytes):
        self.req = req
        self.solver = solver
        self.stream = stream
        self.admitted = admitted
        self.started = started
        self.dt = dt
        self.nbytes = nbytes
        self.queued = 0            # steps enqueued
        self.events = deque()      # (event, steps enqueued after it)


class Server:
    def __init__(self, budget_bytes: int = 120 * 10 ** 9, max_slots: int = 32, chunk: int = 16, device: int = 0,
                 setup_workers: int = 2, clock: Callable[[], float] = time.perf_counter):
        import torch
        self.torch = torch
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.chunk = int(chunk)
        self.device = device
        self.clock = clock
        self.setup_workers = setup_workers
        self.in_use = 0
        self.peak_in_use = 0
        self.max_concurrent = 0
        self.log = []              # (time, event, rid, in_use)
        self.setup_phases = []     # per request: seconds of each set-up phase
        self._lock = threading.Lock()

    def _setup(self, req: SolveRequest, nbytes: int, t0: float) -> _Active:
        torch = self.torch
        torch.cuda.set_device(self.device)
        admitted = self.clock() - t0
        ph = [time.perf_counter()]
        if req.xy is None:
            req.xy, req.tri, req.D_elem = req.build()
        ph.append(time.perf_counter())
        stream = torch.cuda.Stream(device=self.device)
        with torch.cuda.stream(stream):
            s = rdg.Solver(req.xy, req.tri, req.N, req.D_elem, v=req.v, precision=req.precision,
                           device=self.device, stream=stream, interface=req.interface)
            ph.append(time.perf_counter())
            xyn = s.node_coords()
            u0 = np.ascontiguousarray(req.u0(xyn[..., 0], xyn[..., 1]), dtype=s.np_dtype)
            ph.append(time.perf_counter())
            dt = req.dt
            if dt is None:
                dt = 0.5 * SSP_RK3_REAL_EXTENT / spectral_radius(s, torch)
            ph.append(time.perf_counter())
            s.set_state(u0)
            stream.synchronize()
            ph.append(time.perf_counter())
        with self._lock:
            self.setup_phases.append(np.diff(ph))
        return _Active(req, s, stream, admitted, self.clock() - t0, dt, nbytes)

    SETUP_PHASES = ("mesh_build", "library_setup", "initial_state", "step_size", "upload")

    def setup_summary(self):
        """Seconds spent per set-up phase, summed over requests (worker threads overlap)."""
        with self._lock:
            a = np.array(self.setup_phases) if self.setup_phases else np.zeros((0, 5))
        return {n: float(a[:, i].sum()) for i, n in enumerate(self.SETUP_PHASES)}

    def run(self, requests: List[SolveRequest], realtime: bool = True) -> List[SolveResult]:
        """Serve `requests`.  realtime: a request becomes visible at its arrival time on the
        wall clock; otherwise all are visible at once (arrival order kept)."""
        torch = self.torch
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting: deque = deque()
        setting_up = []            # futures
        active: List[_Active] = []
        results: List[SolveResult] = []
        pool = ThreadPoolExecutor(max_workers=self.setup_workers)
        t0 = self.clock()
        try:
            while pending or waiting or setting_up or active:
                now = self.clock() - t0
                while pending and (not realtime or pending[0].arrival <= now):
                    waiting.append(pending.popleft())
                # admission by slots and device memory (reserved before the set-up starts)
                while waiting and len(active) + len(setting_up) < self.max_slots:
                    req = waiting[0]
                    nbytes = request_bytes(req)
                    if nbytes > self.budget:
                        raise ValueError("request %d needs %d bytes, more than the whole budget" % (req.rid, nbytes))
                    if self.in_use + nbytes > self.budget:
                        break
                    waiting.popleft()
                    self.in_use += nbytes
                    self.peak_in_use = max(self.peak_in_use, self.in_use)
                    self.log.append((self.clock() - t0, "admit", req.rid, self.in_use))
                    setting_up.append(pool.submit(self._setup, req, nbytes, t0))
                # requests whose set-up finished join the running mix
                still = []
                for fut in setting_up:
                    if fut.done():
                        active.append(fut.result())
                    else:
                        still.append(fut)
                setting_up = still
                self.max_concurrent = max(self.max_concurrent, len(active))
                # keep up to two chunks queued per resident request
                progressed = False
                for act in active:
                    while act.events and act.events[0][0].query():
                        act.events.popleft()
                    if len(act.events) < 2 and act.queued < act.req.steps:
                        n = min(self.chunk, act.req.steps - act.queued)
                        act.solver.solve_to_time(act.queued * act.dt, act.dt, n)
                        ev = torch.cuda.Event()
                        ev.record(act.stream)
                        act.queued += n
                        act.events.append((ev, act.queued))
                        progressed = True
                # retire requests whose last chunk completed
                keep = []
                for act in active:
                    if act.queued >= act.req.steps and all(e.query() for e, _ in act.events):
                        state = act.solver.get_state_host()
                        act.solver.synchronize()
                        fin = self.clock() - t0
                        results.append(SolveResult(act.req.rid, act.req.arrival, act.admitted, act.started, fin,
                                                   act.solver.K, act.solver.Np, act.req.steps, act.dt, state))
                        act.solver.close()
                        self.in_use -= act.nbytes
                        self.log.append((fin, "finish", act.req.rid, self.in_use))
                        progressed = True
                    else:
                        keep.append(act)
                active = keep
                if not progressed:
                    time.sleep(5e-5)
        finally:
            pool.shutdown(wait=True)
        return results


def solve_alone(req: SolveRequest, dt: float, device: int = 0, precision: Optional[int] = None) -> np.ndarray:
    """The same request on its own (default stream), for checking results in the mix."""
    prec = req.precision if precision is None else precision
    s = rdg.Solver(req.xy, req.tri, req.N, req.D_elem, v=req.v, precision=prec, device=device,
                   interface=req.interface)
    xyn = s.node_coords()
    s.set_state(np.ascontiguousarray(req.u0(xyn[..., 0], xyn[..., 1]), dtype=s.np_dtype))
    s.solve_to_time(0.0, dt, req.steps)
    out = s.get_state_host()
    s.close()
    return out


def latency_stats(results: List[SolveResult]):
    lat = np.array([r.latency for r in results])
    span = max(r.finished for r in results) - min(r.arrival for r in results)
    dofs = sum(r.dof_updates for r in results)
    return {"n": len(results), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "makespan_s": float(span), "gdof_per_s": dofs / span / 1e9}
