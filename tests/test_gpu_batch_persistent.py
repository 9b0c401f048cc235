"""Persistent batch launch (rdg_batch_set_mode RDG_BATCH_PERSISTENT, the default when every
member is FP32 with stored operators and SSP-RK3): one launch per chunk of steps walks a
(member, stage, part, tile) work list over members of orders 1..6 and very different sizes.

* Every member's state after 40 steps (two graph replays of 16-step launches, then eight
  steps in one direct launch) equals its lone solve (the stage and element kernels) to FP32
  rounding (1e-6 element-wise and normwise: the same arithmetic, with order 6's volume term
  on the CUDA cores instead of the tensor cores, and forced members' stage times summed in
  another order) and the branch-graph form of the same batch; a small member follows the
  FP64 oracle.
* Per-order tile mappings (one or two edges per thread, one to four tiles per work item) give
  the same states.
* Bounded waits: with a stage of one member held (a release that never comes) and a 50 ms
  limit, the launch gives up, returns, and the step reports RDG_ETIMEOUT; after the hold is
  removed the batch steps correctly again."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1912_06221_gb300 as rdg
from synth import unit_square_mesh, random_nodal, PERIODIC, DIRICHLET
from oracle.mesh import Mesh
from oracle.rhs import Problem
from tests.test_gpu_parity import parity_err


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


# (N, m, bc, velocity, forced)
SPECS = [(1, 11, PERIODIC, (0.0, 0.0), False),
         (2, 40, PERIODIC, (0.5, 0.25), False),
         (3, 9, DIRICHLET, (0.0, 0.0), True),
         (4, 70, PERIODIC, (-0.3, 0.8), False),
         (5, 13, PERIODIC, (1.0, 0.5), False),
         (6, 17, DIRICHLET, (0.2, 0.0), True),
         (6, 5, PERIODIC, (0.4, -0.2), False),
         (2, 3, PERIODIC, (0.1, 0.1), False)]


def _member(i, N, m, bc, v, forced):
    xy, tri = unit_square_mesh(m, 0.1, 30 + i)
    K = tri.shape[0]
    D = np.where(np.random.default_rng(i).uniform(size=K) < 0.4, 1.0, 0.05)
    s = rdg.Solver(xy, tri, N, D, v=v, bc=bc, period=None if bc == DIRICHLET else (1.0, 1.0), precision=rdg.FP32,
                   interface=rdg.IFACE_ALG1)
    if forced:
        xyn = s.node_coords()
        src = [(np.sin(3 * xyn[..., 0]) * xyn[..., 1], rdg.TAU_COS, 2.0)]
        gh = []
        if s.B:
            g = s.ghost_coords()
            gh = [(g[..., 0] - g[..., 1], rdg.TAU_SIN, 1.0)]
        s.set_forcing(src, gh)
    u0 = np.ascontiguousarray(random_nodal(s.K, s.Np, 50 + i) * 0.1 + 1.0, dtype=np.float32)
    s.set_state(u0)
    h = 1.0 / m
    dt = 0.05 * h * h / (N + 1) ** 4
    return s, u0, dt


def _batch(mode=rdg.BATCH_AUTO, ept=None):
    members = [_member(i, *sp) for i, sp in enumerate(SPECS)]
    b = rdg.Batch(chunk=16)
    b.set_mode(mode)
    if ept:
        for N, (e, tpi) in ept.items():
            b.set_tiles(N, e, tpi)
    for s, u0, dt in members:
        b.add(s, dt, t0=0.25)
    return b, members


def _alone(i):
    s, u0, dt = _member(i, *SPECS[i])
    s.solve_to_time(0.25, dt, 40)
    out = s.get_state_host()
    s.synchronize()
    s.close()
    return out


def test_persistent_batch_equals_alone_and_graph_form():
    b, mem = _batch()
    assert b.mode == rdg.BATCH_PERSISTENT
    b.step(40)
    b.synchronize()
    got = [s.get_state_host() for s, _, _ in mem]
    g, memg = _batch(rdg.BATCH_GRAPH)
    assert g.mode == rdg.BATCH_GRAPH
    g.step(40)
    g.synchronize()
    for i, (s, _, _) in enumerate(memg):
        alone = _alone(i)
        assert parity_err(got[i], alone.astype(np.float64)) < 1e-6, (i, SPECS[i])
        assert parity_err(got[i], s.get_state_host().astype(np.float64)) < 1e-6, (i, SPECS[i])
    for s, _, _ in mem + memg:
        s.close()


def test_persistent_batch_tile_mappings():
    b, mem = _batch(ept={1: (1, 4), 2: (2, 1), 3: (1, 2), 4: (2, 4), 5: (2, 2), 6: (2, 4)})
    b.step(40)
    b.synchronize()
    for i, (s, _, _) in enumerate(mem):
        assert parity_err(s.get_state_host(), _alone(i).astype(np.float64)) < 1e-6, (i, SPECS[i])
        s.close()


def test_persistent_batch_member_follows_oracle():
    xy, tri = unit_square_mesh(6, 0.1, 2)
    K = tri.shape[0]
    D = np.where(np.arange(K) % 3 == 0, 1.0, 0.1)
    s = rdg.Solver(xy, tri, 3, D, v=(0.3, -0.6), precision=rdg.FP32, interface=rdg.IFACE_ALG1)
    big, _, dtb = _member(1, *SPECS[1])
    u0 = (random_nodal(K, s.Np, 3) * 0.2 + 1.0).astype(np.float32)
    s.set_state(u0)
    pr = Problem(Mesh(xy, tri, 3), D, v=(0.3, -0.6), interface="alg1")
    dt = 1e-5
    b = rdg.Batch(chunk=5)
    b.add(s, dt)
    b.add(big, dtb)
    assert b.mode == rdg.BATCH_PERSISTENT
    b.step(12)
    b.synchronize()
    want = pr.solve(u0.astype(np.float64), 0.0, dt, 12)
    assert parity_err(s.get_state_host(), want) < 2e-5
    s.close()
    big.close()


def test_persistent_batch_bounded_wait_times_out():
    b, mem = _batch()
    b.set_wait_limit(0.05)
    b.hold_phase(3, 4)                  # member 3's stage 4 (step 1, stage 1) is never released
    b.step(16)
    with pytest.raises(rdg.RdgError) as e:
        b.synchronize()
    assert e.value.code == rdg.rdg.RDG_ETIMEOUT
    # without the hold the batch steps correctly again from fresh states
    b.hold_phase(-1, -1)
    b.set_wait_limit(1.0)
    for i, (s, u0, dt) in enumerate(mem):
        s.set_state(u0)
    for i, (s, u0, dt) in enumerate(mem):
        b.remove(s)
    for i, (s, u0, dt) in enumerate(mem):
        b.add(s, dt, t0=0.25)
    b.step(40)
    b.synchronize()
    for i, (s, _, _) in enumerate(mem):
        assert parity_err(s.get_state_host(), _alone(i).astype(np.float64)) < 1e-6, (i, SPECS[i])
        s.close()


def test_persistent_mode_refuses_members_that_do_not_fit():
    xy, tri = unit_square_mesh(4, 0.1, 1)
    s64 = rdg.Solver(xy, tri, 2, 1.0, precision=rdg.FP64)
    b = rdg.Batch()
    b.add(s64, 1e-5)
    assert b.mode == rdg.BATCH_GRAPH
    with pytest.raises(rdg.RdgError):
        b.set_mode(rdg.BATCH_PERSISTENT)
    b.remove(s64)
    s64.close()
