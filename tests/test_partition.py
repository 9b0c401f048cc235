"""One mesh split across ranks (paper_1912_06221_gb300/partition.py), on the CPU.

The partition, the halo plan and the per-stage halo exchange are host logic; here they run
with gloo ranks on the CPU, and the stage arithmetic of every rank is the FP64 oracle on its
local mesh (owned + halo elements; oracle/patch.py places them).  Before each SSP-RK3 stage
every rank exchanges the halo rows of the stage input with its neighbours through
torch.distributed point-to-point operations, exactly as the GPU ranks do.  The owned rows of
the split right-hand side and of ten split SSP-RK3 steps equal the unsplit oracle's to
rounding (FP64, 1e-12 relative)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from synth import random_nodal, unit_square_mesh
from paper_1912_06221_gb300.partition import build_plan, face_adjacency, halo_exchange, rcb_partition

N = 3
M = 8
V = (0.7, -0.4)
DT = 4e-5       # 0.45 x the SSP-RK3 stability bound 2.5127 / rho of this problem (rho ~ 2.9e4)


def _case():
    xy, tri = unit_square_mesh(M, 0.1, 5)
    K = tri.shape[0]
    c = xy[tri].mean(axis=1)
    D = np.where(np.hypot(c[:, 0] - 0.5, c[:, 1] - 0.5) < 0.3, 1.0, 0.05)
    return xy, tri, K, D


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle.patch import PatchProblem
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        xy, tri, K, D = _case()
        part = rcb_partition(xy, tri, world)
        plan = build_plan(part, face_adjacency(xy, tri), rank, world)
        owned = plan.elements[: plan.n_owned]
        pp = PatchProblem(xy, tri, N, D, owned, v=V, rings=1, interface="alg1")
        Np = pp.mesh.ops.Np
        send = {p: torch.empty((len(ix), Np), dtype=torch.float64) for p, ix in plan.send.items()}
        recv = {p: torch.empty((n, Np), dtype=torch.float64) for p, (f, n) in plan.recv.items()}

        def L(u_loc, t):
            g = np.zeros((K, Np))
            g[plan.elements] = u_loc            # the patch reads owned and halo rows only
            return pp.rhs(g, t)

        def exchange(u_loc):
            def pack(p, b):
                b.copy_(torch.from_numpy(u_loc[plan.send[p]]))

            def unpack(p, b):
                f, n = plan.recv[p]
                u_loc[f:f + n] = b.numpy()
            halo_exchange(plan, dist, send, recv, pack, unpack)

        u = random_nodal(K, Np, 9)[plan.elements].copy()
        # right-hand side: the local rows come from the global field, halo refreshed first
        u_loc = u.copy()
        u_loc[plan.n_owned:] = 0.0
        exchange(u_loc)
        rhs = L(u_loc, 0.2)
        # ten SSP-RK3 steps, each stage's input halo refreshed before the stage
        dt = DT
        no = plan.n_owned
        for n in range(10):
            t = n * dt
            exchange(u)
            u1 = u.copy()
            u1[:no] = u[:no] + dt * L(u, t)
            exchange(u1)
            u2 = u1.copy()
            u2[:no] = 0.75 * u[:no] + 0.25 * (u1[:no] + dt * L(u1, t + dt))
            exchange(u2)
            u[:no] = u[:no] / 3.0 + 2.0 / 3.0 * (u2[:no] + dt * L(u2, t + 0.5 * dt))
        q.put((rank, owned, rhs, u[:no].copy(), {p: len(ix) for p, ix in plan.send.items()}))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_mesh_rhs_and_steps_equal_unsplit_oracle(world):
    from oracle.mesh import Mesh
    from oracle.rhs import Problem
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    xy, tri, K, D = _case()
    pr = Problem(Mesh(xy, tri, N), D, v=V, interface="alg1")
    u0 = random_nodal(K, pr.mesh.ops.Np, 9)
    want_rhs = pr.rhs(u0, 0.2)
    want_u = pr.solve(u0, 0.0, DT, 10)
    assert np.abs(want_u).max() < 10 * np.abs(u0).max()      # a stable step: nothing grows
    seen = np.zeros(K, bool)
    for rank, owned, rhs, u, sends in res:
        assert not seen[owned].any()
        seen[owned] = True
        assert sends, "every part has a neighbour"
        assert np.abs(rhs - want_rhs[owned]).max() < 1e-12 * np.abs(want_rhs).max()
        assert np.abs(u - want_u[owned]).max() < 1e-12 * np.abs(want_u).max()
    assert seen.all()


def test_partition_plan_is_consistent():
    """Every rank's send list to p holds exactly p's halo block from it, in p's order; the
    halo is the set of other ranks' face neighbours; the parts are balanced."""
    xy, tri, K, D = _case()
    nbr = face_adjacency(xy, tri)
    for world in (2, 3, 4, 5):
        part = rcb_partition(xy, tri, world)
        cnt = np.bincount(part, minlength=world)
        assert cnt.max() - cnt.min() <= 1
        plans = [build_plan(part, nbr, r, world) for r in range(world)]
        for r, pl in enumerate(plans):
            owned = pl.elements[: pl.n_owned]
            halo = set(int(x) for x in nbr[owned].ravel() if part[x] != r)
            assert set(int(x) for x in pl.elements[pl.n_owned:]) == halo
            for p, ix in pl.send.items():
                f, n = plans[p].recv[r]
                assert np.array_equal(pl.elements[ix], plans[p].elements[f:f + n])


class _OracleContext:
    """Stands in for one rank's library context in SplitSolver on the CPU: host tensors for
    the stage buffers, row gathers and scatters by index, and the FP64 oracle as the stage
    arithmetic.  A stage's part 0 records the halo rows it was given; part 1 computes the
    whole stage from the buffer as it is then, so the result is right only if the halo rows
    were refreshed between the parts."""

    def __init__(self, pp, plan, K, u_loc):
        self.pp, self.plan, self.K = pp, plan, K
        self.bufs = [torch.from_numpy(u_loc.copy()), torch.zeros_like(torch.from_numpy(u_loc)),
                     torch.zeros_like(torch.from_numpy(u_loc))]
        self.reg = {}
        for b in self.bufs:
            self.reg[b.data_ptr()] = b
        self.part0_halo = None

    def register(self, t):
        self.reg[t.data_ptr()] = t

    def stage_buffer(self, st):
        return self.bufs[st].data_ptr()

    def rows_gather(self, src, idx, n, dst):
        self.reg[dst][:n] = self.reg[src][idx.long()]

    def rows_scatter(self, src, idx, n, dst):
        self.reg[dst][idx.long()] = self.reg[src][:n]

    def _L(self, u_loc, t):
        g = np.zeros((self.K, u_loc.shape[1]))
        g[self.plan.elements] = u_loc
        return self.pp.rhs(g, t)

    def rk_stage_part(self, st, part, t, dt):
        no = self.plan.n_owned
        src = self.bufs[st]
        if part == 0:
            self.part0_halo = src[no:].clone()
            return
        u, u1, u2 = (b.numpy() for b in self.bufs)
        if st == 0:
            u1[:no] = u[:no] + dt * self._L(u, t)
        elif st == 1:
            u2[:no] = 0.75 * u[:no] + 0.25 * (u1[:no] + dt * self._L(u1, t + dt))
        else:
            u[:no] = u[:no] / 3.0 + 2.0 / 3.0 * (u2[:no] + dt * self._L(u2, t + 0.5 * dt))


def _overlap_worker(rank, world, port, q):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle.patch import PatchProblem
    from paper_1912_06221_gb300.partition import SplitSolver
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        xy, tri, K, D = _case()
        part = rcb_partition(xy, tri, world)
        plan = build_plan(part, face_adjacency(xy, tri), rank, world)
        owned = plan.elements[: plan.n_owned]
        pp = PatchProblem(xy, tri, N, D, owned, v=V, rings=1, interface="alg1")
        Np = pp.mesh.ops.Np
        u_loc = random_nodal(K, Np, 9)[plan.elements].copy()
        u_loc[plan.n_owned:] = 0.0          # halo rows arrive by exchange only
        sp = SplitSolver.__new__(SplitSolver)
        sp.plan = plan
        sp.s = _OracleContext(pp, plan, K, u_loc)
        sp.send_idx = {p: torch.tensor(ix, dtype=torch.int32) for p, ix in plan.send.items()}
        sp.recv_idx = {p: torch.arange(f, f + n, dtype=torch.int32) for p, (f, n) in plan.recv.items()}
        sp.send_bufs = {p: torch.empty((len(ix), Np), dtype=torch.float64) for p, ix in plan.send.items()}
        sp.recv_bufs = {p: torch.empty((n, Np), dtype=torch.float64) for p, (f, n) in plan.recv.items()}
        for b in list(sp.send_bufs.values()) + list(sp.recv_bufs.values()):
            sp.s.register(b)
        stale = 0
        for n in range(10):
            sp.rk_step(n * DT, DT, dist, overlap=True)
            # the halo rows part 0 saw were the previous contents (zero before the first
            # exchange): part 0 ran before the exchange completed
            stale += int(n == 0 and float(sp.s.part0_halo.abs().max()) == 0.0)
        q.put((rank, owned, sp.s.bufs[0].numpy()[: plan.n_owned].copy(), stale))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_split_solver_overlap_steps_equal_unsplit_oracle():
    """SplitSolver.rk_step(overlap=True) on two gloo ranks, the library context replaced by
    the oracle: each stage posts the exchange, runs part 0, waits, stores the halo rows, runs
    part 1; ten steps equal the unsplit oracle's."""
    from oracle.mesh import Mesh
    from oracle.rhs import Problem
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_overlap_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    xy, tri, K, D = _case()
    pr = Problem(Mesh(xy, tri, N), D, v=V, interface="alg1")
    u0 = random_nodal(K, pr.mesh.ops.Np, 9)
    want = pr.solve(u0, 0.0, DT, 10)
    for rank, owned, u, stale in res:
        assert stale == 1
        assert np.abs(u - want[owned]).max() < 1e-12 * np.abs(want).max()
