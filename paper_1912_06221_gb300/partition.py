"""One mesh split across ranks: partition, halo plan and the per-stage halo exchange.

Every edge flux of the method reads all 2 Np nodal values of both elements that share the
edge (the reconstruction on the enclosed parallelogram, Sec. 4 and Algorithm aRDG), not only
their traces.  So a rank that owns part of the mesh needs, before each right-hand-side stage,
the full stage-input rows of the other ranks' elements that touch its own: its halo.  The
rank holds a local mesh of its owned elements followed by its halo elements (grouped by the
owning rank), uploads it with rdg_mesh_upload_partition, and before every stage sends the
rows its neighbours hold as halo and receives its own halo rows (one grouped send/receive per
neighbour per stage, NCCL over torch.distributed on GPUs, gloo on CPUs).  Each rank computes
every local row; the owned rows are exact because the halo rows hold the owners' values.
The exchange overlaps the part of the stage that reads owned rows only (the edges with no
halo side, which the partitioned upload puts first, and the owned volume terms).

Host logic only: the partition (recursive coordinate bisection of element centroids), face
adjacency (vertex ids, then midpoints modulo the period, as the library's mesh upload
matches faces) and the send/receive plan.  The gathers and scatters of rows and every stage
run in the library's kernels (rdg_rows_gather, rdg_rows_scatter, rdg_rk_stage,
rdg_rk_stage_part).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import rdg

FACES = ((0, 1), (1, 2), (2, 0))


def face_adjacency(xy, tri, bc: int = rdg.BC_PERIODIC, period=(1.0, 1.0)):
    """Neighbour element across each face, [K, 3] (-1 where no other face meets it)."""
    xy = np.asarray(xy, np.float64)
    tri = np.asarray(tri, np.int64)
    K = tri.shape[0]
    a = np.concatenate([tri[:, f0] for f0, _ in FACES])       # face i*K + k is face i of k
    b = np.concatenate([tri[:, f1] for _, f1 in FACES])
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    nbr = -np.ones(3 * K, np.int64)
    key = lo * (xy.shape[0] + 1) + hi
    order = np.argsort(key, kind="stable")
    sk = key[order]
    same = np.flatnonzero(sk[1:] == sk[:-1])
    if np.any(np.diff(same) == 1):
        raise ValueError("non-manifold edge")
    nbr[order[same]], nbr[order[same + 1]] = order[same + 1], order[same]
    left = np.flatnonzero(nbr < 0)
    if left.size:
        mid = (xy[a[left]] + xy[b[left]]) / 2
        if bc == rdg.BC_PERIODIC:
            per = np.asarray(period, np.float64)
            mid = np.mod(mid, per)
            mid = np.where(np.abs(mid - per) < 1e-9, 0.0, mid)
            q = np.round(mid * 1e9).astype(np.int64)
        else:
            q = np.round(mid * 1e12).astype(np.int64)
        _, inv, cnt = np.unique(q, axis=0, return_inverse=True, return_counts=True)
        if np.any(cnt > 2):
            raise ValueError("non-manifold edge")
        inv = inv.ravel()
        o = np.argsort(inv, kind="stable")
        si = inv[o]
        pr = np.flatnonzero(si[1:] == si[:-1])
        nbr[left[o[pr]]], nbr[left[o[pr + 1]]] = left[o[pr + 1]], left[o[pr]]
    out = np.where(nbr >= 0, nbr % K, -1)
    return out.reshape(3, K).T.copy()


def rcb_partition(xy, tri, nparts: int):
    """Element owner ranks by recursive coordinate bisection of the centroids: split the
    longer extent at the weighted median, parts in proportion to the ranks on each side."""
    c = np.asarray(xy, np.float64)[np.asarray(tri, np.int64)].mean(axis=1)
    part = np.zeros(c.shape[0], np.int32)

    def split(ids, first, n):
        if n == 1 or ids.size == 0:
            part[ids] = first
            return
        nl = n // 2
        pts = c[ids]
        ax = int(np.argmax(pts.max(axis=0) - pts.min(axis=0)))
        order = ids[np.argsort(pts[:, ax], kind="stable")]
        cut = (ids.size * nl) // n
        split(order[:cut], first, nl)
        split(order[cut:], first + nl, n - nl)

    split(np.arange(c.shape[0]), 0, int(nparts))
    return part


@dataclass
class HaloPlan:
    """One rank's share of a split mesh.  Local element order: the owned elements (ascending
    global id), then the halo elements grouped by owning rank (ascending rank, ascending id).
    send[p]: local indices of the owned rows that rank p holds as halo, in p's order;
    recv[p]: (first local row, count) of the halo block that rank p owns."""
    rank: int
    nparts: int
    elements: np.ndarray
    n_owned: int
    send: Dict[int, np.ndarray] = field(default_factory=dict)
    recv: Dict[int, tuple] = field(default_factory=dict)

    @property
    def peers(self) -> List[int]:
        return sorted(self.recv)


def build_plan(part, nbr, rank: int, nparts: int) -> HaloPlan:
    part = np.asarray(part)
    owned = np.flatnonzero(part == rank)
    nb = nbr[owned]                                    # [n_owned, 3]
    cand = np.unique(nb[nb >= 0])
    halo_all = cand[part[cand] != rank]
    recv, blocks = {}, []
    first = owned.size
    for p in range(nparts):
        if p == rank:
            continue
        hp = halo_all[part[halo_all] == p]              # ascending global ids
        if hp.size:
            recv[p] = (first, int(hp.size))
            blocks.append(hp)
            first += hp.size
    elements = np.concatenate([owned] + blocks) if blocks else owned
    send = {}
    for p in recv:
        # rank p's halo block from this rank: this rank's elements next to p's, ascending ids
        mine_next = owned[np.any((nb >= 0) & (part[np.maximum(nb, 0)] == p), axis=1)]
        send[p] = np.searchsorted(owned, mine_next).astype(np.int32)
    return HaloPlan(rank, nparts, elements, int(owned.size), send, recv)


def halo_exchange(plan: HaloPlan, dist, send_bufs, recv_bufs, pack, unpack, group=None):
    """One halo exchange: pack(p, buf) fills the rows for every neighbour p, one grouped
    send/receive per neighbour (torch.distributed point-to-point), unpack(p, buf) stores the
    received halo block.  A rank with no neighbour does nothing."""
    for p in plan.peers:
        pack(p, send_bufs[p])
    ops = [dist.P2POp(dist.isend, send_bufs[p], p, group) for p in plan.peers]
    ops += [dist.P2POp(dist.irecv, recv_bufs[p], p, group) for p in plan.peers]
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()
    for p in plan.peers:
        unpack(p, recv_bufs[p])


class SplitSolver:
    """One rank's part of a mesh split across ranks, on its GPU: the library context of the
    local mesh (owned + halo triangles) and the device buffers of its halo exchange."""

    def __init__(self, xy, tri, N, D_elem, plan: HaloPlan, v=(0.0, 0.0), bc=rdg.BC_PERIODIC, period=(1.0, 1.0),
                 precision=rdg.FP32, device=0, interface=rdg.IFACE_ALG1, stream=None):
        import torch
        self.torch = torch
        self.plan = plan
        tri_l = np.asarray(tri)[plan.elements]
        D = np.broadcast_to(np.asarray(D_elem, np.float64), (np.asarray(tri).shape[0],))[plan.elements]
        self.s = rdg.Solver(xy, tri_l, N, D, v=v, bc=bc, period=period, precision=precision, device=device,
                            stream=stream, interface=interface, n_owned=plan.n_owned)
        dev = "cuda:%d" % device
        self.send_idx = {p: torch.tensor(ix, dtype=torch.int32, device=dev) for p, ix in plan.send.items()}
        self.recv_idx = {p: torch.arange(f, f + n, dtype=torch.int32, device=dev) for p, (f, n) in plan.recv.items()}
        self.send_bufs = {p: torch.empty((ix.size, self.s.Np), dtype=self.s.dtype, device=dev)
                          for p, ix in plan.send.items()}
        self.recv_bufs = {p: torch.empty((n, self.s.Np), dtype=self.s.dtype, device=dev)
                          for p, (f, n) in plan.recv.items()}

    @property
    def n_owned(self):
        return self.plan.n_owned

    def pack(self, src: int, p: int, buf):
        """Rows of `src` (device address of a local [K, Np] array) that rank p holds as halo."""
        self.s.rows_gather(src, self.send_idx[p], self.send_idx[p].numel(), buf.data_ptr())

    def unpack(self, dst: int, p: int, buf):
        """Received rows of rank p into the halo rows of `dst`."""
        self.s.rows_scatter(buf.data_ptr(), self.recv_idx[p], self.recv_idx[p].numel(), dst)

    def exchange(self, dst: int, dist, group=None):
        """Halo rows of the local array at device address dst from their owners."""
        halo_exchange(self.plan, dist, self.send_bufs, self.recv_bufs,
                      lambda p, b: self.pack(dst, p, b), lambda p, b: self.unpack(dst, p, b), group)

    def exchange_begin(self, dst: int, dist, group=None):
        """Pack the rows every neighbour needs from the local array at dst and post the grouped
        send/receive; returns the requests (on NCCL the transfers run on NCCL's stream)."""
        for p in self.plan.peers:
            self.pack(dst, p, self.send_bufs[p])
        ops = [dist.P2POp(dist.isend, self.send_bufs[p], p, group) for p in self.plan.peers]
        ops += [dist.P2POp(dist.irecv, self.recv_bufs[p], p, group) for p in self.plan.peers]
        return dist.batch_isend_irecv(ops) if ops else []

    def exchange_end(self, reqs, dst: int):
        """Wait for the requests (the solver's stream waits for NCCL) and store the halo rows."""
        for r in reqs:
            r.wait()
        for p in self.plan.peers:
            self.unpack(dst, p, self.recv_bufs[p])

    def rk_step(self, t: float, dt: float, dist, group=None, stages: int = 3, overlap: bool = True):
        """One step.  overlap: each stage's exchange runs while the edges with no halo side
        and the owned volume terms are computed (rdg_rk_stage_part 0), the rest after it
        (part 1); otherwise the halo rows are refreshed before each whole stage."""
        for st in range(stages):
            buf = self.s.stage_buffer(st)
            if overlap:
                reqs = self.exchange_begin(buf, dist, group)
                self.s.rk_stage_part(st, 0, t, dt)
                self.exchange_end(reqs, buf)
                self.s.rk_stage_part(st, 1, t, dt)
            else:
                self.exchange(buf, dist, group)
                self.s.rk_stage(st, t, dt)

    def set_owned_state(self, u_global):
        """Resident state from a global [K_global, Np] array (owned and halo rows)."""
        self.s.set_state(np.ascontiguousarray(np.asarray(u_global)[self.plan.elements], self.s.np_dtype))

    def owned_state(self):
        return self.s.get_state_host()[: self.plan.n_owned]
