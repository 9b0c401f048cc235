"""FP32 consistency properties of the stored operators and the stage update.

* A constant is a steady solution of the heat equation and the reconstruction reproduces it
  (Sec. 2.3: polynomials up to degree N are recovered exactly, so their gradient is exact);
  with v = 0 every FP32 and FP64 step keeps a constant state bit for bit.  This pins the
  difference form of the flux and volume operators (the constant enters only through the
  exactly zero upwind row sum) and the increment form of the SSP-RK3 combinations (whose
  FP32 coefficients would otherwise sum to 1 + 3e-8 and scale the state every step).
* Adding a constant offset to the state changes the FP32 right-hand side error (against the
  oracle on the same rounded input) by no more than a small factor: the large diffusive
  entries multiply differences of nearby values, not the values themselves.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1912_06221_gb300 as rdg
from synth import unit_square_mesh, random_nodal, PERIODIC
from oracle.mesh import Mesh
from oracle.rhs import Problem


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("N", [1, 3, 4, 6])
@pytest.mark.parametrize("prec", [rdg.FP32, rdg.FP64])
@pytest.mark.parametrize("iface", [rdg.IFACE_ALG2, rdg.IFACE_HARMONIC])
def test_constant_state_is_kept_exactly(N, prec, iface):
    xy, tri = unit_square_mesh(10, 0.15, 4)
    K = tri.shape[0]
    D = np.where(np.random.default_rng(2).uniform(size=K) < 0.5, 1.0, 1e-3)
    s = rdg.Solver(xy, tri, N, D, v=(0.0, 0.0), precision=prec, interface=iface)
    c = 0.7310585786300049
    u0 = np.full((K, s.Np), c, dtype=s.np_dtype)
    s.set_state(u0)
    h = 0.1
    dt = 0.1 * h * h / (N + 1) ** 4
    s.solve_to_time(0.0, dt, 37)          # two graph replays and five direct steps
    got = s.get_state_host()
    assert np.array_equal(got, u0)
    r = torch.empty((K, s.Np), dtype=s.dtype, device="cuda")
    s.rhs_eval(torch.tensor(u0, device="cuda"), r, 0.0)
    s.synchronize()
    assert float(r.abs().max()) == 0.0
    s.close()


@pytest.mark.parametrize("N", [2, 4, 6])
def test_fp32_rhs_error_does_not_grow_with_an_offset(N):
    xy, tri = unit_square_mesh(9, 0.1, 5)
    K = tri.shape[0]
    D = np.where(np.random.default_rng(5).uniform(size=K) < 0.4, 1.0, 0.05)
    v = (0.3, -0.2)
    s = rdg.Solver(xy, tri, N, D, v=v, precision=rdg.FP32)
    me = Mesh(xy, tri, N)
    pr = Problem(me, D, v=v)
    f = np.sin(2 * np.pi * me.x) * np.cos(2 * np.pi * me.y) + 0.01 * random_nodal(K, s.Np, 6)
    errs = []
    for off in (0.0, 16.0):
        u32 = (f + off).astype(np.float32)
        ud = torch.tensor(u32, device="cuda")
        rd = torch.empty_like(ud)
        s.rhs_eval(ud, rd, 0.0)
        s.synchronize()
        want = pr.rhs(u32.astype(np.float64))
        errs.append(np.linalg.norm(rd.cpu().numpy() - want) / np.linalg.norm(pr.rhs(f)))
    # the offset's rounding of the input is in `want`; what is left is the arithmetic's
    assert errs[1] < 4 * errs[0] + 1e-6, errs
    s.close()
