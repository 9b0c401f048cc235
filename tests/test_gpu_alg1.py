"""The paper's Algorithm 1 in the library (RDG_IFACE_ALG1) against the oracle: the per-edge
FP64 operators built on the GPU edge by edge (the oracle's flux_algorithm1 applied to unit
vectors), the right-hand side in FP64 and FP32 with a 1e4 contrast in D, SSP-RK3 steps, and
the GEMM-form precision mode falling back to the stored operators for this rule."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1912_06221_gb300 as rdg
from synth import unit_square_mesh, random_nodal, PERIODIC, DIRICHLET
from oracle.mesh import Mesh
from oracle.rhs import Problem, stable_dt

from tests.test_gpu_parity import TOL, parity_err, relerr


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _case(N, bc, prec=rdg.FP64, m=7, seed=5):
    xy, tri = unit_square_mesh(m, 0.12, seed)
    K = tri.shape[0]
    D = np.where(np.random.default_rng(seed).uniform(size=K) < 0.4, 1.0, 1e-4)
    v = (0.6, -0.35)
    s = rdg.Solver(xy, tri, N, D, v=v, bc=bc, precision=prec, interface=rdg.IFACE_ALG1)
    me = Mesh(xy, tri, N, bc=bc)
    return s, me, D, v


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("bc", [PERIODIC, DIRICHLET])
def test_alg1_edge_operators_match_oracle(N, bc):
    s, me, D, v = _case(N, bc)
    W, ids = s.edge_operators()
    pr = Problem(me, D, v=v, ghost_fn=(lambda x, y, t: 0 * x), interface="alg1")
    eo, ops = pr.eops, me.ops
    Np, Nfp, E = ops.Np, ops.Nfp, me.E
    # oracle operator of every edge, column by column: [u1; u2] = unit vector j
    Op = np.zeros((E, Nfp, 2 * Np))
    for j in range(2 * Np):
        u1 = np.zeros((E, Np))
        u2 = np.zeros((E, Np))
        (u1 if j < Np else u2)[:, j % Np] = 1.0
        Op[:, :, j] = eo.flux_algorithm1(eo.reconstruct(u1, u2), pr.D1e, pr.D2e)
    key = {(k1, f1): e for e, (k1, f1, k2, f2, _, _) in enumerate(me.edges)}
    for el in range(s.E):
        k1, f1, k2, f2 = ids[el]
        e = key.get((k1, f1))
        swapped = e is None
        if swapped:
            e = key[(k2, f2)]
        Jf = me.sJ[me.edges[e][0], me.edges[e][1]]
        Wo = -Jf * Op[e]
        vn = eo.n1[e] @ pr.v
        for i in range(Nfp):
            if vn >= 0:
                Wo[i, ops.Fmask[me.edges[e][1]][i]] += Jf * vn
            else:
                f2o = me.edges[e][3] if me.edges[e][2] >= 0 else 1
                Wo[i, Np + ops.Fmask[f2o][Nfp - 1 - i]] += Jf * vn
        if swapped:
            Wo = -Wo[::-1][:, np.r_[Np:2 * Np, 0:Np]]
        scale = np.abs(Wo).max()
        assert np.abs(W[el] - Wo).max() < 1e-11 * scale, (el, np.abs(W[el] - Wo).max() / scale)
    s.close()


@pytest.mark.parametrize("N", [1, 3, 4, 6])
@pytest.mark.parametrize("prec", [rdg.FP64, rdg.FP32, rdg.FP32_3XTF32])
def test_alg1_rhs_parity(N, prec):
    s, me, D, v = _case(N, DIRICHLET, prec=prec, m=9)
    g = s.ghost_coords()
    s.set_forcing([], [(np.cos(g[..., 0]) + g[..., 1], rdg.TAU_SIN, 2.0)])
    pr = Problem(me, D, v=v, ghost_fn=lambda x, y, t: (np.cos(x) + y) * np.sin(2.0 * t), interface="alg1")
    u = random_nodal(s.K, s.Np, 12)
    if prec != rdg.FP64:
        u = u.astype(np.float32).astype(np.float64)
    ud = torch.tensor(u, dtype=s.dtype, device="cuda")
    rd = torch.empty_like(ud)
    s.rhs_eval(ud, rd, 0.4)
    s.synchronize()
    tol = TOL[rdg.FP64] if prec == rdg.FP64 else TOL[rdg.FP32]
    assert parity_err(rd.cpu().numpy(), pr.rhs(u, 0.4)) < tol
    s.close()


@pytest.mark.parametrize("prec", [rdg.FP64, rdg.FP32])
def test_alg1_rk_steps(prec):
    s, me, D, v = _case(3, PERIODIC, prec=prec, m=6)
    pr = Problem(me, D, v=v, interface="alg1")
    u0 = random_nodal(s.K, s.Np, 3) * 0.1 + np.sin(2 * np.pi * me.x)
    if prec == rdg.FP32:
        u0 = u0.astype(np.float32).astype(np.float64)
    dt = stable_dt(pr, 0.4, 20)
    s.set_state(u0)
    s.solve_to_time(0.0, dt, 21)
    got = s.get_state_host()
    s.synchronize()
    assert parity_err(got, pr.solve(u0, 0.0, dt, 21)) < (1e-10 if prec == rdg.FP64 else 2e-5)
    s.close()
