"""One mesh split across ranks on the GPU (library path: rdg_mesh_upload_partition,
rdg_rk_stage, rdg_stage_buffer, rdg_rows_gather / rdg_rows_scatter).

Every run here has one GPU, so the ranks are emulated in one process: one library context
per part on the same GPU, and the transport between them (NCCL point-to-point between GPUs)
replaced by device-to-device copies of the packed halo rows, made before every stage in
the order a grouped send/receive would.  No kernel of one part waits on another part's
kernel.  The owned rows after ten split SSP-RK3 steps equal the unsplit oracle's (FP64
1e-10, FP32 1e-5, normwise and element by element) and the unsplit library run's, with each
stage run whole after the exchange or in two parts around it (rdg_rk_stage_part: the edges
with no halo side and the owned volume terms before the exchange, the rest after); the
partitioned upload puts a multiple of 32 halo-free edges first."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1912_06221_gb300 as rdg
from paper_1912_06221_gb300.partition import SplitSolver, build_plan, face_adjacency, rcb_partition
from synth import random_nodal, unit_square_mesh
from oracle.mesh import Mesh
from oracle.rhs import Problem, stable_dt


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _err(a, b):
    d = np.asarray(a, float) - b
    return max(np.abs(d).max() / np.abs(b).max(), np.linalg.norm(d) / np.linalg.norm(b))


def _exchange_all(parts, stage):
    """The halo exchange of every part for `stage`, in one process: pack, copy, unpack."""
    for sp in parts:
        buf = sp.s.stage_buffer(stage)
        for p in sp.plan.peers:
            sp.pack(buf, p, sp.send_bufs[p])
    for r, sp in enumerate(parts):
        for p in sp.plan.peers:
            sp.recv_bufs[p].copy_(parts[p].send_bufs[r])
    for sp in parts:
        buf = sp.s.stage_buffer(stage)
        for p in sp.plan.peers:
            sp.unpack(buf, p, sp.recv_bufs[p])


# order 3 in every combination; order 6 (where FP32 runs each stage whole in part 1) on two
# ranks with periodic boundaries, both precisions, whole and two-part stages
CASES = ([(w, p, bc, ov, 3) for w in (2, 3) for p in (rdg.FP64, rdg.FP32)
          for bc in (rdg.BC_PERIODIC, rdg.BC_DIRICHLET) for ov in (False, True)]
         + [(2, p, rdg.BC_PERIODIC, ov, 6) for p in (rdg.FP64, rdg.FP32) for ov in (False, True)])


@pytest.mark.parametrize("world,prec,bc,overlap,N", CASES)
def test_split_mesh_steps_equal_unsplit(world, prec, bc, overlap, N):
    m, v = (16, (0.7, -0.4)) if N == 3 else (8, (0.7, -0.4))
    xy, tri = unit_square_mesh(m, 0.1, 6)
    K = tri.shape[0]
    c = xy[tri].mean(axis=1)
    D = np.where(np.hypot(c[:, 0] - 0.5, c[:, 1] - 0.5) < 0.3, 1.0, 0.05)
    per = (1.0, 1.0) if bc == rdg.BC_PERIODIC else None
    part = rcb_partition(xy, tri, world)
    nbr = face_adjacency(xy, tri, bc, per or (1.0, 1.0))
    plans = [build_plan(part, nbr, r, world) for r in range(world)]
    parts = [SplitSolver(xy, tri, N, D, pl, v=v, bc=bc, period=per, precision=prec) for pl in plans]
    whole = rdg.Solver(xy, tri, N, D, v=v, bc=bc, period=per, precision=prec, interface=rdg.IFACE_ALG1)
    u0 = random_nodal(K, whole.Np, 4)
    if prec == rdg.FP32:
        u0 = u0.astype(np.float32).astype(np.float64)
    for sp in parts:
        sp.set_owned_state(u0)
    whole.set_state(u0)
    me = Mesh(xy, tri, N, bc=bc)
    pr = Problem(me, D, v=v, interface="alg1", ghost_fn=(lambda x, y, t: 0.0 * x) if bc == rdg.BC_DIRICHLET else None)
    dt, nsteps = stable_dt(pr, 0.5, 20), 10
    for sp in parts:
        n_owned, e_split = sp.s.split_counts()
        assert n_owned == sp.n_owned and e_split % 32 == 0
        _, ids = sp.s.edge_operators()
        k1, k2 = ids[:e_split, 0], ids[:e_split, 2]
        assert (k1 < n_owned).all() and (k2 < n_owned).all()
        assert (np.maximum(ids[e_split:, 0], ids[e_split:, 2]) >= n_owned).sum() > 0
        if N == 3:
            assert e_split > 0
    for n in range(nsteps):
        for st in range(3):
            if overlap:
                for sp in parts:
                    sp.s.rk_stage_part(st, 0, n * dt, dt)
                _exchange_all(parts, st)
                for sp in parts:
                    sp.s.rk_stage_part(st, 1, n * dt, dt)
            else:
                _exchange_all(parts, st)
                for sp in parts:
                    sp.s.rk_stage(st, n * dt, dt)
    whole.solve_to_time(0.0, dt, nsteps)
    got = np.zeros((K, whole.Np))
    for sp in parts:
        got[sp.plan.elements[: sp.n_owned]] = sp.owned_state()
        sp.s.synchronize()
    want = pr.solve(u0, 0.0, dt, nsteps)
    assert np.abs(want).max() < 10 * np.abs(u0).max()      # a stable step: nothing grows
    tol = 1e-10 if prec == rdg.FP64 else 1e-5
    assert _err(got, want) < tol
    assert _err(got, whole.get_state_host()) < tol
    for sp in parts:
        assert sp.plan.peers and sp.s.B >= 0
        sp.s.close()
    whole.close()


def test_rows_gather_scatter_and_index_check():
    xy, tri = unit_square_mesh(4, 0.1, 1)
    s = rdg.Solver(xy, tri, 2, 1.0, precision=rdg.FP64)
    u = torch.tensor(random_nodal(s.K, s.Np, 1), device="cuda")
    idx = torch.tensor([5, 0, 31, 7], dtype=torch.int32, device="cuda")
    out = torch.zeros((4, s.Np), dtype=torch.float64, device="cuda")
    s.rows_gather(u.data_ptr(), idx, 4, out.data_ptr())
    back = torch.zeros_like(u)
    s.rows_scatter(out.data_ptr(), idx, 4, back.data_ptr())
    s.synchronize()
    assert torch.equal(out, u[idx.long()])
    assert torch.equal(back[idx.long()], u[idx.long()])
    # an index outside the rows is skipped and reported, not accessed
    bad = torch.tensor([1, s.K + 3], dtype=torch.int32, device="cuda")
    s.rows_gather(u.data_ptr(), bad, 2, out.data_ptr())
    with pytest.raises(rdg.RdgError):
        s.synchronize()
    s.close()


def test_partition_upload_rejects_unmatched_owned_face():
    """A periodic part whose owned triangles leave a face unmatched is refused."""
    xy, tri = unit_square_mesh(4, 0.1, 1)
    with pytest.raises(rdg.RdgError) as e:
        rdg.Solver(xy, tri[:10], 2, 1.0, n_owned=10)
    assert e.value.code == rdg.rdg.RDG_EMESH


@pytest.mark.parametrize("prec", [rdg.FP64, rdg.FP32])
def test_stage_parts_on_an_unsplit_context(prec):
    """A context uploaded whole: part 0 enqueues nothing, part 1 the whole stage, so parts 0
    then 1 of every stage equal rdg_rk_step; a part other than 0 or 1 is refused."""
    xy, tri = unit_square_mesh(8, 0.1, 2)
    D = np.where(np.arange(tri.shape[0]) % 4 == 0, 1.0, 0.1)
    a = rdg.Solver(xy, tri, 2, D, v=(0.3, 0.2), precision=prec)
    b = rdg.Solver(xy, tri, 2, D, v=(0.3, 0.2), precision=prec)
    assert a.split_counts() == (a.K, a.E)
    u0 = random_nodal(a.K, a.Np, 3)
    a.set_state(u0)
    b.set_state(u0)
    dt = 1e-5
    for n in range(4):
        a.rk_step(n * dt, dt)
        for st in range(3):
            b.rk_stage_part(st, 0, n * dt, dt)
            b.rk_stage_part(st, 1, n * dt, dt)
    assert np.array_equal(a.get_state_host(), b.get_state_host())
    with pytest.raises(rdg.RdgError):
        b.rk_stage_part(0, 2, 0.0, dt)
    a.close()
    b.close()
