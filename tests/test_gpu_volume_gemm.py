"""GPU: the order-6 FP32 volume term formed as a tensor-core GEMM (tcgen05, split 3xTF32).

Parity with the FP64 oracle on meshes of one ragged element tile and of several tiles with a
ragged tail, through every integrator stage kind; then, on a mesh of 157 element tiles (more
than one per persistent block on 152 SMs, so the blocks loop and prefetch), agreement with
the FP64 library path, which the parity tests pin to the oracle at every order.  Tolerance:
FP32 rounding over rows of ~100 terms, 1e-5 normwise and element-wise as for the other
FP32 forms.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1912_06221_gb300 as rdg
from synth import unit_square_mesh, random_nodal, PERIODIC, DIRICHLET
from oracle.mesh import Mesh
from oracle.rhs import Problem


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


from tests.test_gpu_parity import parity_err  # noqa: E402  (normwise and element-wise)


def _solver(m, prec, bc=PERIODIC, seed=7, v=(0.6, -0.3)):
    xy, tri = unit_square_mesh(m, 0.1, seed)
    K = tri.shape[0]
    D = np.where(np.random.default_rng(seed).uniform(size=K) < 0.4, 0.8, 0.05)
    return rdg.Solver(xy, tri, 6, D, v=v, bc=bc, precision=prec), xy, tri, D


def _rhs(s, u, t=0.0):
    ud = torch.tensor(u, dtype=s.dtype, device="cuda")
    rd = torch.empty_like(ud)
    s.rhs_eval(ud, rd, t)
    s.synchronize()
    return rd.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("m,bc", [(6, PERIODIC), (20, DIRICHLET)])
def test_order6_fp32_rhs_matches_oracle(m, bc):
    """72 elements (one ragged tile); 800 elements (7 tiles, 32 in the last)."""
    s, xy, tri, D = _solver(m, rdg.FP32, bc)
    me = Mesh(xy, tri, 6, bc=bc)
    pr = Problem(me, D, v=(0.6, -0.3), ghost_fn=(lambda x, y, t: 0 * x))
    u = random_nodal(s.K, s.Np, 5).astype(np.float32).astype(np.float64)
    assert parity_err(_rhs(s, u), pr.rhs(u)) < 1e-5
    s.close()


@pytest.mark.parametrize("integrator", [rdg.SSP_RK3, rdg.LSRK54])
def test_order6_fp32_steps_match_oracle(integrator):
    s, xy, tri, D = _solver(8, rdg.FP32)
    s.set_integrator(integrator)
    me = Mesh(xy, tri, 6, bc=PERIODIC)
    pr = Problem(me, D, v=(0.6, -0.3))
    u0 = random_nodal(s.K, s.Np, 9).astype(np.float32).astype(np.float64)
    dt, n = 2e-6, 7
    s.set_state(torch.tensor(u0, dtype=torch.float32, device="cuda"))
    s.solve_to_time(0.0, dt, n)
    got = s.get_state_host().astype(np.float64)
    want = pr.solve(u0, 0.0, dt, n, scheme="ssp3" if integrator == rdg.SSP_RK3 else "lsrk54")
    assert parity_err(got, want) < 1e-5
    s.close()


def test_order6_fp32_many_tiles_agrees_with_fp64_path():
    """20000 elements = 157 tiles of 128: the persistent blocks take a second tile."""
    s32, _, _, _ = _solver(100, rdg.FP32, seed=11)
    s64, _, _, _ = _solver(100, rdg.FP64, seed=11)
    u = random_nodal(s32.K, s32.Np, 13).astype(np.float32).astype(np.float64)
    r32, r64 = _rhs(s32, u), _rhs(s64, u)
    assert parity_err(r32, r64) < 1e-5
    # the tail tile's rows and a middle tile's are as accurate as the whole
    for sl in (slice(156 * 128, None), slice(77 * 128, 78 * 128)):
        assert parity_err(r32[sl], r64[sl]) < 1e-5
    s32.synchronize()   # raises if a kernel self-check fired
    s32.close()
    s64.close()


def test_volume_gemm_bounded_wait_times_out_and_recovers():
    """Bounded wait of the order-6 volume kernel: with one element tile's MMAs never issued
    (test hook), its block's completion wait gives up (1 s, once more for 1 s), the block
    leaves and frees its tensor memory, and the next synchronize reports RDG_ETIMEOUT; with
    the hold removed the context evaluates the right-hand side against the oracle again."""
    xy, tri = unit_square_mesh(12, 0.1, 4)         # 288 triangles: 3 element tiles, the last ragged
    K = tri.shape[0]
    D = np.where(np.arange(K) % 5 == 0, 1.0, 0.1)
    s = rdg.Solver(xy, tri, 6, D, v=(0.4, -0.3), precision=rdg.FP32)
    pr = Problem(Mesh(xy, tri, 6), D, v=(0.4, -0.3))
    u = random_nodal(K, s.Np, 8).astype(np.float32).astype(np.float64)
    ud = torch.tensor(u, dtype=torch.float32, device="cuda")
    rd = torch.empty_like(ud)
    s.gemm_hold_tile(1)
    s.rhs_eval(ud, rd, 0.0)
    with pytest.raises(rdg.RdgError) as e:
        s.synchronize()
    assert e.value.code == rdg.rdg.RDG_ETIMEOUT
    s.gemm_hold_tile(-1)
    s.rhs_eval(ud, rd, 0.0)
    s.synchronize()
    assert parity_err(rd.double().cpu().numpy(), pr.rhs(u, 0.0)) < 1e-5
    s.close()
