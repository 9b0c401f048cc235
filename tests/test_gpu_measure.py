"""GPU measurement entry points: the FP64 error norms against the oracle's, and the FMA rates.

The library's error norms (Eqs. L2_norm_cellUnit, Linf_norm_cellUnit) use a collapsed Gauss
rule with N + 3 points per direction; the oracle's (oracle.refops.triangle_quadrature) uses
N + 4.  Both are exact for total degree 2N + 4,
so on errors whose square (and, for the cell means, whose absolute value) is a polynomial of
that degree they agree to rounding."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1912_06221_gb300 as rdg
from synth import random_nodal, unit_square_mesh
from oracle.mesh import Mesh
from oracle.rhs import error_norms


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("N", [1, 2, 4, 6])
@pytest.mark.parametrize("prec", [rdg.FP64, rdg.FP32])
def test_error_norms_match_oracle(N, prec):
    xy, tri = unit_square_mesh(7, 0.1, 2)
    s = rdg.Solver(xy, tri, N, 1.0, precision=prec)
    me = Mesh(xy, tri, N)
    q = s.error_quadrature()
    assert q.shape == (s.K, (N + 3) ** 2, 2)
    # zero field against a positive polynomial of degree 2: e^2 and |e| are polynomials
    ue = lambda x, y, t: 1.0 + x * x + 0.5 * y * y + 0.25 * x * y
    z = torch.zeros((s.K, s.Np), dtype=s.dtype, device="cuda")
    l2, li = s.error_norms(ue(q[..., 0], q[..., 1], 0.0), z)
    o2, oi = error_norms(me, np.zeros((s.K, s.Np)), ue, 0.0)
    assert abs(l2 - o2) < 1e-12 * o2 and abs(li - oi) < 1e-12 * oi
    # a random nodal field against zero: e is the field itself (degree N), e^2 of degree 2N
    u = random_nodal(s.K, s.Np, 4)
    ud = torch.tensor(u, dtype=s.dtype, device="cuda")
    zero = lambda x, y, t: 0.0 * x
    l2, _ = s.error_norms(np.zeros(q.shape[:2]), ud)
    o2, _ = error_norms(me, ud.double().cpu().numpy(), zero, 0.0)
    assert abs(l2 - o2) < 1e-12 * o2
    # the resident state is used when no field is given
    s.set_state(ud)
    assert s.error_norms(np.zeros(q.shape[:2]))[0] == l2
    s.close()


def test_fma_rates():
    f32 = rdg.peak_fma(0, rdg.FP32)
    f64 = rdg.peak_fma(0, rdg.FP64)
    # GB300: 152 SMs x 128 FP32 lanes x 2 FLOP x ~2 GHz ~ 78 TFLOP/s; FP64 far below
    assert 2e13 < f32 < 2e14, f32
    assert 0 < f64 < f32, (f32, f64)


def test_stream_read_bandwidth():
    """A 1 GiB streaming read reaches a sizeable share of the HBM rate; a 64 MiB read, a
    standalone launch with its fixed ramp-up, a smaller one."""
    t_big = rdg.stream_read_seconds(0, 1 << 30)
    t_small = rdg.stream_read_seconds(0, 64 << 20)
    bw_big = (1 << 30) / t_big
    bw_small = (64 << 20) / t_small
    assert 2e12 < bw_big < 9e12, bw_big
    assert bw_small < bw_big
