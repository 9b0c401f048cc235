"""The paper's five-stage fourth-order low-storage Runge-Kutta scheme in the library
(rdg_set_integrator(RDG_INTEGRATOR_LSRK54)) against the oracle, and the paper's own
verification problems (Sec. 5.1 Gaussian diffusion, Sec. 5.2 advection-diffusion) on the
GPU over the paper's grid-a series (32 .. 8192 triangles; stand-ins with every triangle pair
a parallelogram), time step fixed by the finest mesh as in the paper: the observed L2 order
between the two finest meshes is within 0.3 of Tables purediff_ooa / adv_diff_ooa for P1 and
P3, and between P and P + 1 for P2 (the paper states O(h^P) for even P)."""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1912_06221_gb300 as rdg
from synth import paper_gaussian, unit_square_mesh, random_nodal, DIRICHLET
from oracle.mesh import Mesh
from oracle.rhs import Problem, stable_dt, error_norms

from tests.test_gpu_parity import _forcing, parity_err, relerr
from tests.test_oracle_paper_problems import _table


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("N", [2, 4])
@pytest.mark.parametrize("prec", [rdg.FP64, rdg.FP32])
def test_lsrk_steps_and_graph_match_oracle(N, prec):
    xy, tri = unit_square_mesh(7, 0.1, 3)
    K = tri.shape[0]
    D = np.where(np.random.default_rng(3).uniform(size=K) < 0.3, 1.0, 0.02)
    s = rdg.Solver(xy, tri, N, D, v=(0.7, -0.4), bc=DIRICHLET, precision=prec)
    s.set_integrator(rdg.LSRK54)
    me = Mesh(xy, tri, N, bc=DIRICHLET)
    osrc, gfn = _forcing(s, me)
    pr = Problem(me, D, v=(0.7, -0.4), source=osrc, ghost_fn=gfn)
    u0 = random_nodal(s.K, s.Np, 5) * 0.1 + me.x
    if prec == rdg.FP32:
        u0 = u0.astype(np.float32).astype(np.float64)
    dt = stable_dt(pr, 0.4, 20)
    t0 = 0.125
    s.set_state(u0)
    for n in range(3):
        s.rk_step(t0 + n * dt, dt)
    got = s.get_state_host()
    want = pr.solve(u0, t0, dt, 3, scheme="lsrk54")
    assert parity_err(got, want) < (1e-11 if prec == rdg.FP64 else 1e-5)
    s.set_state(u0)
    s.solve_to_time(t0, dt, 21)      # one graph chunk of 16 steps and 5 direct steps
    got = s.get_state_host()
    s.synchronize()
    want = pr.solve(u0, t0, dt, 21, scheme="lsrk54")
    assert parity_err(got, want) < (1e-10 if prec == rdg.FP64 else 2e-5)
    s.close()


def _gpu_errors(N, advection, ms, dt_mesh):
    """L2 errors at t = 0.5 on each mesh (FP64 GPU), dt from the power iteration of the
    oracle-free GPU operator of the finest mesh."""
    T = 0.5
    w = paper_gaussian(dt_mesh, N, advection=advection)
    s = rdg.Solver(w.xy, w.tri, N, w.D_elem, v=w.v, period=(10.0, 10.0), precision=rdg.FP64)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((s.K, s.Np), generator=g, device="cuda", dtype=torch.float64)
    y = torch.empty_like(x)
    for _ in range(40):
        x /= torch.linalg.vector_norm(x)
        s.rhs_eval(x, y, 0.0)
        x, y = y, x
    rho = float(torch.linalg.vector_norm(x))
    s.close()
    n = int(math.ceil(T / (0.5 * 2.5127 / rho)))
    dt = T / n
    errs = []
    for m in ms:
        w = paper_gaussian(m, N, advection=advection)
        s = rdg.Solver(w.xy, w.tri, N, w.D_elem, v=w.v, period=(10.0, 10.0), precision=rdg.FP64)
        s.set_integrator(rdg.LSRK54)
        xyn = s.node_coords()
        s.set_state(w.exact(xyn[..., 0], xyn[..., 1], 0.0))
        s.solve_to_time(0.0, dt, n)
        u = s.get_state_host()
        s.synchronize()
        me = Mesh(w.xy, w.tri, N, period=(10.0, 10.0))
        errs.append(error_norms(me, u, w.exact, T)[0])
        s.close()
    return errs, dt, n


@pytest.mark.parametrize("advection", [False, True])
def test_paper_problem_small_meshes_match_oracle(advection):
    """GPU (FP64, LSRK) and oracle on the 32- and 128-triangle meshes with the same dt."""
    N, T = 2, 0.5
    wl = [paper_gaussian(m, N, advection=advection) for m in (4, 8)]
    prs = [Problem(Mesh(w.xy, w.tri, N, period=(10.0, 10.0)), w.D_elem, v=w.v) for w in wl]
    dt = stable_dt(prs[-1], 0.5, 30)
    n = int(math.ceil(T / dt))
    dt = T / n
    for w, pr in zip(wl, prs):
        me = pr.mesh
        want = pr.solve(w.exact(me.x, me.y, 0.0), 0.0, dt, n, scheme="lsrk54")
        s = rdg.Solver(w.xy, w.tri, N, w.D_elem, v=w.v, period=(10.0, 10.0), precision=rdg.FP64)
        s.set_integrator(rdg.LSRK54)
        s.set_state(w.exact(me.x, me.y, 0.0))
        s.solve_to_time(0.0, dt, n)
        got = s.get_state_host()
        s.synchronize()
        s.close()
        assert parity_err(got, want) < 1e-10


@pytest.mark.parametrize("N", [1, 2, 3])
@pytest.mark.parametrize("advection,table", [(False, "purediff_ooa.txt"), (True, "advdiff_ooa.txt")])
def test_paper_problem_orders_full_grid_a_series(N, advection, table):
    ms = (4, 8, 16, 32, 64)                  # 32, 128, 512, 2048, 8192 triangles
    errs, dt, n = _gpu_errors(N, advection, ms, ms[-1])
    assert all(errs[i] > errs[i + 1] for i in range(len(ms) - 1)), errs
    order = math.log2(errs[-2] / errs[-1])
    if N % 2:
        paper = _table(table)["a"][N - 1]
        assert abs(order - paper) < 0.3, (N, advection, order, paper, errs)
    else:
        # even P: the paper's conclusions state O(h^P) convergence for even P (citing Oden et
        # al.), between P and the P + 1 of odd orders; its table's P2 entry (about 2.8) comes
        # from its own mesh levels, and on this series the order approaches P
        assert N - 0.2 < order < N + 1.2, (N, advection, order, errs)
