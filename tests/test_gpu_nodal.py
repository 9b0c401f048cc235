"""GPU: a spatially varying D given at the nodes (rdg_operator_setup_nodal; Sec. 3, D a
function of space in Eq. NDG_diffusion_once_matrixForm_reference_general, with Algorithms 1
and 2) against the FP64 oracle: every order, every interface rule, periodic and Dirichlet
with sources and ghost data, a random positive nodal D that jumps between elements.
Tolerances as for the scalar parity tests (normwise and element by element): one right-hand
side FP64 1e-12, FP32 1e-5; a state after many steps FP64 1e-10, FP32 2e-5."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1912_06221_gb300 as rdg
from synth import unit_square_mesh, random_nodal, PERIODIC, DIRICHLET
from oracle.mesh import Mesh
from oracle.rhs import Problem, stable_dt
from tests.test_gpu_parity import _forcing, parity_err

IF = {rdg.IFACE_ALG1: "alg1", rdg.IFACE_ALG2: "alg2", rdg.IFACE_HARMONIC: "harmonic"}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _nodal_D(K, Np, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.05, 1.0, (K, 1)) * rng.uniform(0.5, 1.5, (K, Np))


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("iface", [rdg.IFACE_ALG1, rdg.IFACE_ALG2, rdg.IFACE_HARMONIC])
@pytest.mark.parametrize("prec", [rdg.FP64, rdg.FP32])
def test_nodal_rhs_parity(N, iface, prec):
    for bc in (PERIODIC, DIRICHLET):
        xy, tri = unit_square_mesh(8, 0.1, 3)
        Np = (N + 1) * (N + 2) // 2
        D = _nodal_D(tri.shape[0], Np, 5 + N)
        s = rdg.Solver(xy, tri, N, D, v=(0.7, -0.4), bc=bc, period=None if bc == DIRICHLET else (1.0, 1.0),
                       precision=prec, interface=iface)
        me = Mesh(xy, tri, N, bc=bc)
        osrc, gfn = _forcing(s, me, with_src=True, with_ghost=(bc == DIRICHLET))
        pr = Problem(me, D, v=(0.7, -0.4), source=osrc, ghost_fn=gfn, interface=IF[iface])
        u = random_nodal(s.K, s.Np, 13)
        ud = torch.tensor(u, dtype=s.dtype, device="cuda")
        rd = torch.empty_like(ud)
        s.rhs_eval(ud, rd, 0.37)
        s.synchronize()
        want = pr.rhs(ud.double().cpu().numpy(), 0.37)
        assert parity_err(rd.cpu().numpy(), want) < (1e-12 if prec == rdg.FP64 else 1e-5), (bc,)
        s.close()


@pytest.mark.parametrize("prec", [rdg.FP64, rdg.FP32])
def test_nodal_steps_and_graph_replay(prec):
    N = 4
    xy, tri = unit_square_mesh(8, 0.1, 4)
    D = _nodal_D(tri.shape[0], 15, 2)
    s = rdg.Solver(xy, tri, N, D, v=(0.3, 0.5), precision=prec, interface=rdg.IFACE_ALG1)
    pr = Problem(Mesh(xy, tri, N), D, v=(0.3, 0.5), interface="alg1")
    u0 = random_nodal(s.K, s.Np, 5) * 0.1 + pr.mesh.x
    if prec == rdg.FP32:
        u0 = u0.astype(np.float32).astype(np.float64)
    dt = stable_dt(pr, 0.4, 20)
    s.set_state(u0)
    s.solve_to_time(0.0, dt, 21)
    got = s.get_state_host()
    s.synchronize()
    assert parity_err(got, pr.solve(u0, 0.0, dt, 21)) < (1e-10 if prec == rdg.FP64 else 2e-5)
    s.close()


def test_constant_nodal_D_equals_element_D_and_static_entry_refuses():
    xy, tri = unit_square_mesh(7, 0.1, 2)
    K = tri.shape[0]
    d = np.random.default_rng(1).uniform(0.1, 1.0, K)
    u = torch.tensor(random_nodal(K, 28, 4), dtype=torch.float64, device="cuda")
    res = []
    for iface in (rdg.IFACE_ALG1, rdg.IFACE_ALG2):
        for D in (d, np.repeat(d[:, None], 28, axis=1)):
            s = rdg.Solver(xy, tri, 6, D, v=(0.2, 0.1), precision=rdg.FP64, interface=iface)
            r = torch.empty_like(u)
            s.rhs_eval(u, r, 0.0)
            s.synchronize()
            res.append(r.cpu().numpy())
            if D.ndim == 2:
                lib = rdg.load()
                rc = lib.rdg_rhs_eval_static(s.ctx, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(r.data_ptr()), 0.0)
                assert rc == rdg.rdg.RDG_ESTATE
            s.close()
    assert parity_err(res[1], res[0]) < 1e-12
    assert parity_err(res[3], res[2]) < 1e-12
