"""The GEMM form of the edge flux (RDG_FP32_3XTF32: tcgen05 split-3xTF32 products against the
order's reference matrices) against the FP64 oracle, element by element, on meshes that span
several 128-edge tiles with a ragged last tile, periodic and Dirichlet, with forcing; and
against the stored-operator FP32 path on the same inputs.

Tolerance: normwise relative 1e-5 for one right-hand side and 2e-5 after 21 steps, as for
FP32 (the split products carry about 21 significant bits per product, below FP32 rounding
of the accumulation).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1912_06221_gb300 as rdg
from synth import unit_square_mesh, random_nodal, PERIODIC, DIRICHLET
from oracle.mesh import Mesh
from oracle.rhs import Problem, stable_dt

from tests.test_gpu_parity import _forcing, parity_err, relerr

TF = rdg.FP32_3XTF32


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _pair(N, m, bc, seed=3, v=(0.7, -0.4)):
    xy, tri = unit_square_mesh(m, 0.1, seed)
    K = tri.shape[0]
    D = np.where(np.random.default_rng(seed).uniform(size=K) < 0.3, 1.0, 0.02)
    s = rdg.Solver(xy, tri, N, D, v=v, bc=bc, precision=TF)
    me = Mesh(xy, tri, N, bc=bc)
    return s, me, D, xy, tri


def _rhs(s, u, t):
    ud = torch.tensor(u, dtype=torch.float32, device="cuda")
    rd = torch.empty_like(ud)
    s.rhs_eval(ud, rd, t)
    s.synchronize()
    return rd.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("bc", [PERIODIC, DIRICHLET])
def test_rhs_parity_tf32(N, bc):
    s, me, D, _, _ = _pair(N, 11, bc)          # 242 triangles, 2 edge tiles for periodic
    osrc, gfn = _forcing(s, me, with_src=True, with_ghost=(bc == DIRICHLET))
    pr = Problem(me, D, v=(0.7, -0.4), source=osrc, ghost_fn=gfn)
    u = random_nodal(s.K, s.Np, 11)
    u32 = u.astype(np.float32).astype(np.float64)
    got = _rhs(s, u32, 0.37)
    assert parity_err(got, pr.rhs(u32, 0.37)) < 1e-5
    s.close()


@pytest.mark.parametrize("N", [3, 4, 5])
def test_tf32_matches_stored_operator_fp32_larger_mesh(N):
    """21x21x2 Dirichlet mesh: 1323 edges (11 tiles, ragged) and 882 elements (7 volume
    tiles): the GEMM form and the stored-operator FP32 path agree."""
    xy, tri = unit_square_mesh(21, 0.1, 9)
    K = tri.shape[0]
    D = np.where(np.random.default_rng(9).uniform(size=K) < 0.5, 1.0, 1e-3)
    a = rdg.Solver(xy, tri, N, D, v=(0.3, 0.9), bc=DIRICHLET, precision=TF)
    b = rdg.Solver(xy, tri, N, D, v=(0.3, 0.9), bc=DIRICHLET, precision=rdg.FP32)
    for s in (a, b):
        g = s.ghost_coords()
        s.set_forcing([], [(np.sin(g[..., 0]) * g[..., 1], rdg.TAU_CONST, 0.0)])
    u = random_nodal(K, a.Np, 4).astype(np.float32).astype(np.float64)
    ra, rb = _rhs(a, u, 0.0), _rhs(b, u, 0.0)
    assert parity_err(ra, rb) < 1e-5
    me = Mesh(xy, tri, N, bc=DIRICHLET)
    pr = Problem(me, D, v=(0.3, 0.9), ghost_fn=lambda x, y, t: np.sin(x) * y)
    assert parity_err(ra, pr.rhs(u, 0.0)) < 1e-5
    a.close()
    b.close()


@pytest.mark.parametrize("N", [2, 4])
def test_tf32_rk_steps_and_graph(N):
    s, me, D, _, _ = _pair(N, 7, DIRICHLET)
    osrc, gfn = _forcing(s, me)
    pr = Problem(me, D, v=(0.7, -0.4), source=osrc, ghost_fn=gfn)
    u0 = (random_nodal(s.K, s.Np, 5) * 0.1 + me.x).astype(np.float32).astype(np.float64)
    dt = stable_dt(pr, 0.4, 20)
    s.set_state(u0)
    s.solve_to_time(0.125, dt, 21)
    got = s.get_state_host()
    s.synchronize()
    assert parity_err(got, pr.solve(u0, 0.125, dt, 21)) < 2e-5
    s.close()


def test_tf32_order6_uses_stored_operators_and_static_entry_rejects():
    s, me, D, _, _ = _pair(6, 5, PERIODIC)
    pr = Problem(me, D, v=(0.7, -0.4))
    u = random_nodal(s.K, s.Np, 2).astype(np.float32).astype(np.float64)
    assert parity_err(_rhs(s, u, 0.0), pr.rhs(u)) < 1e-5
    # order 6 keeps stored operators, so the allocation-free entry point accepts it
    ud6 = torch.tensor(u, dtype=torch.float32, device="cuda")
    rd6 = torch.empty_like(ud6)
    s._call("rdg_rhs_eval_static", rdg.rdg._P(ud6.data_ptr()), rdg.rdg._P(rd6.data_ptr()), 0.0)
    s.synchronize()
    assert parity_err(rd6.cpu().numpy(), pr.rhs(u)) < 1e-5
    s.close()
    s4, _, _, _, _ = _pair(4, 5, PERIODIC)
    ud = torch.zeros((s4.K, s4.Np), dtype=torch.float32, device="cuda")
    rd = torch.empty_like(ud)
    with pytest.raises(rdg.RdgError) as e:
        s4._call("rdg_rhs_eval_static", rdg.rdg._P(ud.data_ptr()), rdg.rdg._P(rd.data_ptr()), 0.0)
    assert e.value.code == rdg.rdg.RDG_ESTATE
    s4.close()


def test_tf32_constant_state_kept_exactly():
    xy, tri = unit_square_mesh(10, 0.15, 4)
    K = tri.shape[0]
    D = np.where(np.random.default_rng(2).uniform(size=K) < 0.5, 1.0, 1e-3)
    for N in (1, 3, 5):
        s = rdg.Solver(xy, tri, N, D, v=(0.0, 0.0), precision=TF)
        u0 = np.full((K, s.Np), 0.7310586, dtype=np.float32)
        s.set_state(u0)
        s.solve_to_time(0.0, 1e-6, 19)
        assert np.array_equal(s.get_state_host(), u0)
        s.synchronize()
        s.close()


@pytest.mark.parametrize("tile", [0, 3])
def test_gemm_form_bounded_wait_times_out_and_recovers(tile):
    """Bounded waits of the warp-specialised GEMM kernel: with one edge tile never released
    by its producer (test hook), the epilogue's wait for it gives up after 1 s, the CTA aborts
    its other roles' waits, drains its MMAs and frees its tensor memory, and the next
    synchronize reports RDG_ETIMEOUT; with the hold removed the same context evaluates the
    right-hand side correctly again."""
    s, me, D, _, _ = _pair(4, 24, PERIODIC)     # 1152 triangles, 1728 edges: 14 edge tiles
    pr = Problem(me, D, v=(0.7, -0.4))
    u = random_nodal(s.K, s.Np, 5).astype(np.float32).astype(np.float64)
    ud = torch.tensor(u, dtype=torch.float32, device="cuda")
    rd = torch.empty_like(ud)
    s.gemm_hold_tile(tile)
    s.rhs_eval(ud, rd, 0.0)
    with pytest.raises(rdg.RdgError) as e:
        s.synchronize()
    assert e.value.code == rdg.rdg.RDG_ETIMEOUT
    s.gemm_hold_tile(-1)
    assert parity_err(_rhs(s, u, 0.0), pr.rhs(u, 0.0)) < 1e-5
    s.close()
