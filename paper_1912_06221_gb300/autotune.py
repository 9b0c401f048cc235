"""Measured per-order choices for batched and served FP32 solves.

For each order N the library has two FP32-accurate edge-flux forms: the stored per-edge
operators (RDG_FP32, an HBM-bound GEMV) and the GEMM form on the tensor cores
(RDG_FP32_3XTF32, N <= 5).  Which is faster depends on the order and the problem size, so
the tuner times both on the caller's own problem (a few replayed stages after a warm-up) and
caches the winner per (device, N, size class).  The graph chunk of a batch (steps per
replayed graph) is tuned the same way on the batch itself, and so is the persistent batch
launch's tile mapping per order (edges per thread of an edge work item) and the batch form
(persistent launch or branch graph).  All timing is CUDA events on the solver's or batch's
stream; nothing here computes the method.
"""
from __future__ import annotations

import math
from typing import Dict, Iterable, List, Optional, Tuple

import numpy as np

from . import rdg

_cache: Dict[Tuple[int, int, int], dict] = {}


def size_class(n_triangles: int) -> int:
    """Problems within a factor of 4 in size share a decision."""
    return int(math.floor(math.log(max(n_triangles, 1), 4)))


def _time_steps(torch, solver, u0, dt, steps, reps=3):
    solver.set_state(u0)
    solver.solve_to_time(0.0, dt, steps)        # warm-up (and graph capture)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        solver.set_state(u0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(solver.stream)
        solver.solve_to_time(0.0, dt, steps)
        b.record(solver.stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def choose_precision(xy, tri, N: int, D_elem, v=(0.0, 0.0), dt: float = 1e-9, device: int = 0,
                     steps: int = 16, **solver_kw) -> dict:
    """Fastest FP32-accurate form for this problem's (device, N, size class): returns
    {"precision": rdg.FP32 or rdg.FP32_3XTF32, "ms": {...}, "cached": bool}.  The first
    problem of a class is timed (both forms, `steps` replayed steps each); later ones reuse
    the decision."""
    import torch
    key = (device, N, size_class(len(tri)))
    if key in _cache:
        return dict(_cache[key], cached=True)
    cands = [rdg.FP32] + ([rdg.FP32_3XTF32] if N <= 5 else [])
    ms = {}
    for prec in cands:
        s = rdg.Solver(xy, tri, N, D_elem, v=v, precision=prec, device=device, **solver_kw)
        u0 = torch.zeros((s.K, s.Np), dtype=torch.float32, device="cuda:%d" % device)
        ms[prec] = _time_steps(torch, s, u0, dt, steps)
        s.synchronize()
        s.close()
    best = min(ms, key=ms.get)
    _cache[key] = {"precision": best, "ms": {("fp32" if p == rdg.FP32 else "fp32_3xtf32"): t for p, t in ms.items()}}
    return dict(_cache[key], cached=False)


def choose_chunk(batch, members: List, u0s: List, steps: int, candidates: Iterable[int] = (5, 10, 25, 50)) -> dict:
    """Steps per replayed graph for this batch: each candidate is timed on one batch step of
    `steps` steps (members reset to their initial states before each run); returns the best
    and every time.  The batch is left with the best chunk."""
    import torch
    times = {}
    for c in candidates:
        batch.set_chunk(c)
        for s, u in zip(members, u0s):
            s.set_state(u)
        batch.step(steps)                  # capture and warm up
        torch.cuda.synchronize()
        for s, u in zip(members, u0s):
            s.set_state(u)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(batch.stream)
        batch.step(steps)
        b.record(batch.stream)
        torch.cuda.synchronize()
        times[c] = a.elapsed_time(b)
    best = min(times, key=times.get)
    batch.set_chunk(best)
    return {"chunk": best, "ms": times}


def _time_batch(torch, batch, members, u0s, steps):
    for s, u in zip(members, u0s):
        s.set_state(u)
    batch.step(steps)                      # capture and warm up
    torch.cuda.synchronize()
    for s, u in zip(members, u0s):
        s.set_state(u)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(batch.stream)
    batch.step(steps)
    b.record(batch.stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def choose_tiles(batch, members: List, u0s: List, steps: int) -> dict:
    """Per-order tile mapping of the persistent batch launch: for every order present, one
    or two edges per thread of an edge tile and one, two or four tiles per work item, chosen
    one order at a time (the others kept at their best so far) by timing the batch itself.  Then the batch form (the persistent
    launch or the branch graph) by timing both.  The batch is left with the best choices;
    returns them and every time."""
    import torch
    orders = sorted({s.N for s in members})
    times = {}
    best = {}
    if batch.mode != rdg.BATCH_PERSISTENT:
        return {"mode": "graph", "edges_per_thread_tiles_per_item": {}, "ms": {}}
    for N in orders:
        tN = {}
        for e in (1, 2):                       # edges per thread, one tile per item
            batch.set_tiles(N, e, 1)
            tN[(e, 1)] = _time_batch(torch, batch, members, u0s, steps)
        e = min((1, 2), key=lambda x: tN[(x, 1)])
        for tpi in (2, 4):                     # then tiles per item
            batch.set_tiles(N, e, tpi)
            tN[(e, tpi)] = _time_batch(torch, batch, members, u0s, steps)
        best[N] = min(tN, key=tN.get)
        batch.set_tiles(N, *best[N])
        times["N%d" % N] = {"%d edges/thread, %d tiles/item" % k: v for k, v in tN.items()}
    # the last order's best time was taken with every order at its best
    t_pers = min(times["N%d" % orders[-1]].values())
    batch.set_mode(rdg.BATCH_GRAPH)
    t_graph = _time_batch(torch, batch, members, u0s, steps)
    mode = "persistent" if t_pers <= t_graph else "graph"
    batch.set_mode(rdg.BATCH_AUTO if mode == "persistent" else rdg.BATCH_GRAPH)
    times["persistent"] = t_pers
    times["graph"] = t_graph
    return {"mode": mode, "edges_per_thread_tiles_per_item": {N: list(v) for N, v in best.items()}, "ms": times}
