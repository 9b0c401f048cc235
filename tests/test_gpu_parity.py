"""GPU parity: the sm_103a library through its C ABI against the FP64 oracle.

Meshes span several kernel tiles with a ragged tail (128-element blocks, 32-edge tiles):
m = 9 gives 162 triangles and 243 edges.  Every comparison with the oracle is both normwise
(relative L2) and element by element (the largest pointwise difference over max |oracle|),
with one tolerance for both: FP64 <= 1e-12 for one right-hand side, <= 1e-10 for a state
after many steps; FP32 <= 1e-5 (rounding of O(1e-7) per operation accumulated over the few
hundred terms of a row, well inside 1e-5).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1912_06221_gb300 as rdg
from synth import unit_square_mesh, random_nodal, PERIODIC, DIRICHLET, heat_sin_mode
from oracle.mesh import Mesh
from oracle.rhs import Problem, stable_dt

TOL = {rdg.FP64: 1e-12, rdg.FP32: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - b) / max(np.linalg.norm(b), 1e-300))


def parity_err(a, b):
    """The larger of the normwise relative L2 error and the element-wise error, the largest
    |a - b| over every element and node divided by max |b|: a wrong value confined to a few
    elements or to one face slot moves the element-wise error long before the normwise one."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    ew = float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
    return max(relerr(a, b), ew)


def _setup(N, m=9, seed=3, bc=PERIODIC, prec=rdg.FP64, v=(0.7, -0.4), varD=True, jitter=0.1):
    xy, tri = unit_square_mesh(m, jitter, seed)
    K = tri.shape[0]
    D = np.where(np.random.default_rng(seed).uniform(size=K) < 0.3, 1.0, 0.02) if varD else np.full(K, 0.5)
    s = rdg.Solver(xy, tri, N, D, v=v, bc=bc, precision=prec)
    me = Mesh(xy, tri, N, bc=bc)
    return s, me, D


GF = [(lambda x, y: np.sin(np.pi * x) * np.cos(2 * np.pi * y), rdg.TAU_COS, 1.0),
      (lambda x, y: 0.3 * x * y + 0.1, rdg.TAU_SIN, 2.0)]
SF = [(lambda x, y: np.cos(3 * x) * y, rdg.TAU_CONST, 0.0), (lambda x, y: x - y * y, rdg.TAU_SIN, 5.0)]


def _tau(kind, om, t):
    return 1.0 if kind == rdg.TAU_CONST else (math.cos(om * t) if kind == rdg.TAU_COS else math.sin(om * t))


def _forcing(s, me, with_src=True, with_ghost=True):
    """Install the same separable source/ghost data on both sides (each at its own nodes)."""
    xyn = s.node_coords()
    src = [(f(xyn[..., 0], xyn[..., 1]), k, o) for f, k, o in SF] if with_src else []
    gh = []
    if with_ghost and s.B:
        gxy = s.ghost_coords()
        gh = [(f(gxy[..., 0], gxy[..., 1]), k, o) for f, k, o in GF]
    s.set_forcing(src, gh)
    osrc = [(f(me.x, me.y), k, o) for f, k, o in SF] if with_src else []
    gfn = (lambda x, y, t: sum(f(x, y) * _tau(k, o, t) for f, k, o in GF)) if with_ghost else None
    return osrc, gfn


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("prec", [rdg.FP64, rdg.FP32])
def test_node_coords_match_oracle(N, prec):
    s, me, D = _setup(N, prec=prec)
    xy = s.node_coords()
    assert np.abs(xy[..., 0] - me.x).max() < 1e-14 and np.abs(xy[..., 1] - me.y).max() < 1e-14


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("bc", [PERIODIC, DIRICHLET])
def test_edge_operators_match_oracle(N, bc):
    """Per-edge FP64 flux operators built on the GPU equal the oracle's composition
    J_f ( -D~ n1.grad(reconstruction) + upwind ) edge by edge."""
    s, me, D = _setup(N, bc=bc)
    W, ids = s.edge_operators()
    pr = Problem(me, D, v=(0.7, -0.4), ghost_fn=(lambda x, y, t: 0 * x))
    eo = pr.eops
    ops = me.ops
    key = {}
    for e, (k1, f1, k2, f2, _, _) in enumerate(me.edges):
        key[(k1, f1)] = e
    Np, Nfp = ops.Np, ops.Nfp
    for el in range(s.E):
        k1, f1, k2, f2 = ids[el]
        e = key.get((k1, f1))
        swapped = False
        if e is None:
            e = key[(k2, f2)]
            swapped = True
        # oracle operator: g = n1.grad u~ as a linear map of [u1; u2]
        Rx, Ry, Sx, Sy = eo.Rx[e]
        n1 = eo.n1[e]
        G = (n1[0] * Rx + n1[1] * Ry) * ops.DR + (n1[0] * Sx + n1[1] * Sy) * ops.DS
        Op = G @ ops.Apinv @ np.block([[eo.P1[e], np.zeros((Np, Np))], [np.zeros((Np, Np)), eo.P2[e]]])
        Jf = me.sJ[me.edges[e][0], me.edges[e][1]]
        Wo = -Jf * pr.Dt[e][:, None] * Op
        vn = n1 @ pr.v
        for i in range(Nfp):
            if vn >= 0:
                Wo[i, ops.Fmask[me.edges[e][1]][i]] += Jf * vn
            else:
                f2o = me.edges[e][3] if me.edges[e][2] >= 0 else 1
                Wo[i, Np + ops.Fmask[f2o][Nfp - 1 - i]] += Jf * vn
        if swapped:   # the library took the other element as side 1: flux negated, reversed
            Wo = -Wo[::-1][:, np.r_[Np:2 * Np, 0:Np]]
        scale = np.abs(Wo).max()
        assert np.abs(W[el] - Wo).max() < 1e-11 * scale, (el, np.abs(W[el] - Wo).max() / scale)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("prec", [rdg.FP64, rdg.FP32])
@pytest.mark.parametrize("bc", [PERIODIC, DIRICHLET])
def test_rhs_parity(N, prec, bc):
    s, me, D = _setup(N, prec=prec, bc=bc)
    osrc, gfn = _forcing(s, me, with_src=True, with_ghost=(bc == DIRICHLET))
    pr = Problem(me, D, v=(0.7, -0.4), source=osrc, ghost_fn=gfn)
    u = random_nodal(s.K, s.Np, 11)
    ud = torch.tensor(u, dtype=s.dtype, device="cuda")
    rd = torch.empty_like(ud)
    t = 0.37
    s.rhs_eval(ud, rd, t)
    s.synchronize()
    want = pr.rhs(u.astype(np.float32).astype(np.float64) if prec == rdg.FP32 else u, t)
    assert parity_err(rd.cpu().numpy(), want) < TOL[prec]


@pytest.mark.parametrize("N", [1, 3, 5])
@pytest.mark.parametrize("prec", [rdg.FP64, rdg.FP32])
def test_rhs_parity_harmonic_interface(N, prec):
    xy, tri = unit_square_mesh(9, 0.1, 3)
    D = np.where(np.random.default_rng(3).uniform(size=tri.shape[0]) < 0.3, 1.0, 1e-4)
    s = rdg.Solver(xy, tri, N, D, v=(0.7, -0.4), precision=prec, interface=rdg.IFACE_HARMONIC)
    me = Mesh(xy, tri, N)
    pr = Problem(me, D, v=(0.7, -0.4), interface="harmonic")
    u = random_nodal(s.K, s.Np, 8)
    ud = torch.tensor(u, dtype=s.dtype, device="cuda")
    rd = torch.empty_like(ud)
    s.rhs_eval(ud, rd, 0.0)
    s.synchronize()
    want = pr.rhs(u.astype(np.float32).astype(np.float64) if prec == rdg.FP32 else u)
    assert parity_err(rd.cpu().numpy(), want) < TOL[prec]


@pytest.mark.parametrize("N", [2, 4, 6])
@pytest.mark.parametrize("prec", [rdg.FP64, rdg.FP32])
def test_rk_steps_and_graph_replay(N, prec):
    """Direct SSP-RK3 steps and the CUDA-graph replay (a chunk of 16 steps plus a remainder)
    both follow the oracle, with time-dependent sources and Dirichlet ghosts."""
    s, me, D = _setup(N, prec=prec, bc=DIRICHLET, m=7)
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
    want = pr.solve(u0, t0, dt, 3)
    assert parity_err(got, want) < (1e-11 if prec == rdg.FP64 else 1e-5)
    s.set_state(u0)
    s.solve_to_time(t0, dt, 21)
    got = s.get_state_host()
    want = pr.solve(u0, t0, dt, 21)
    assert parity_err(got, want) < (1e-10 if prec == rdg.FP64 else 2e-5)


def test_heat_sin_mode_fp64_full_run():
    """N = 2, 16x16x2 jittered periodic mesh, 200 steps at dt = 0.1 h^2/(D (N+1)^4): the GPU
    FP64 state equals the oracle's, and both decay at the exact rate exp(-8 pi^2 D t)."""
    w = heat_sin_mode()
    s = rdg.Solver(w.xy, w.tri, w.N, w.D_elem, precision=rdg.FP64)
    xyn = s.node_coords()
    u0 = w.u0(xyn[..., 0], xyn[..., 1])
    s.set_state(u0)
    s.solve_to_time(0.0, w.dt, w.steps)
    got = s.get_state_host()
    me = Mesh(w.xy, w.tri, w.N)
    pr = Problem(me, w.D_elem)
    want = pr.solve(w.u0(me.x, me.y), 0.0, w.dt, w.steps)
    assert parity_err(got, want) < 1e-10
    T = w.steps * w.dt
    Mw = me.J[:, None] * (u0 @ me.ops.M)
    rate = math.log(np.sum(Mw * got) / np.sum(Mw * u0)) / (-8 * math.pi ** 2 * T)
    assert abs(rate - 1) < 1e-2


def test_conservation_and_constants_on_gpu():
    s, me, D = _setup(4, m=12, prec=rdg.FP64)
    ur = torch.tensor(random_nodal(s.K, s.Np, 2), device="cuda")
    r = torch.empty_like(ur)
    s.rhs_eval(ur, r, 0.0)
    s.synchronize()
    opnorm = float(r.abs().max() / ur.abs().max())      # scale of the operator's rows
    u = torch.full((s.K, s.Np), 1.75, dtype=torch.float64, device="cuda")
    rc = torch.empty_like(u)
    s.rhs_eval(u, rc, 0.0)
    s.synchronize()
    assert float(rc.abs().max()) < 1e-13 * opnorm * 1.75      # L 1 = 0 to rounding
    tot = np.sum(me.J[:, None] * (r.cpu().numpy() @ me.ops.M))
    scale = np.sum(np.abs(me.J[:, None] * (r.cpu().numpy() @ me.ops.M)))
    assert abs(tot) < 1e-12 * scale


def test_error_paths():
    xy, tri = unit_square_mesh(3, 0.1, 0)
    bad = tri.copy()
    bad[0] = bad[0][::-1]          # clockwise triangle
    with pytest.raises(rdg.RdgError) as ei:
        rdg.Solver(xy, bad, 2, 1.0)
    assert ei.value.code == -4
    with pytest.raises(rdg.RdgError) as ei:
        rdg.Solver(xy, tri, 7, 1.0)
    assert ei.value.code == -1
    with pytest.raises(rdg.RdgError) as ei:
        rdg.Solver(xy, tri, 2, -1.0)
    assert ei.value.code == -1
    # a periodic mesh that is not periodic (Dirichlet-style hole): drop one triangle
    with pytest.raises(rdg.RdgError) as ei:
        rdg.Solver(xy, tri[1:], 2, 1.0)
    assert ei.value.code == -4
    s = rdg.Solver(xy, tri, 2, 1.0)
    with pytest.raises(ValueError):
        s.rhs_eval(torch.zeros(3, device="cuda"), torch.zeros(3, device="cuda"))


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("prec", [rdg.FP64, rdg.FP32])
def test_rhs_parity_larger_mesh(N, prec):
    """20x20x2 Dirichlet mesh: 1200 edges (38 edge tiles) and 800 elements (7 element tiles,
    interleaved with the edge tiles in the stage kernel's grid)."""
    s, me, D = _setup(N, m=20, prec=prec, bc=DIRICHLET)
    osrc, gfn = _forcing(s, me)
    pr = Problem(me, D, v=(0.7, -0.4), source=osrc, ghost_fn=gfn)
    u = random_nodal(s.K, s.Np, 21)
    ud = torch.tensor(u, dtype=s.dtype, device="cuda")
    rd = torch.empty_like(ud)
    s.rhs_eval(ud, rd, 0.2)
    s.synchronize()
    want = pr.rhs(u.astype(np.float32).astype(np.float64) if prec == rdg.FP32 else u, 0.2)
    assert parity_err(rd.cpu().numpy(), want) < TOL[prec]


@pytest.mark.parametrize("prec", [rdg.FP32, rdg.FP64])
def test_repeatable_at_scale(prec):
    """A 160x160x2 mesh (76800 edges): repeated right-hand sides and a graph-replayed solve are
    bitwise repeatable and no kernel self-check fires."""
    xy, tri = unit_square_mesh(160, 0.1, 5)
    s = rdg.Solver(xy, tri, 4, 0.3, v=(0.2, 0.1), precision=prec)
    u = torch.tensor(random_nodal(s.K, s.Np, 3), dtype=s.dtype, device="cuda")
    r1, r2 = torch.empty_like(u), torch.empty_like(u)
    s.rhs_eval(u, r1, 0.0)
    for _ in range(20):
        s.rhs_eval(u, r2, 0.0)
    s.synchronize()
    assert torch.equal(r1, r2)
    s.set_state(u)
    s.solve_to_time(0.0, 1e-9, 40)
    a = s.get_state_host()
    s.set_state(u)
    s.solve_to_time(0.0, 1e-9, 40)
    b = s.get_state_host()
    s.synchronize()
    assert np.array_equal(a, b) and np.isfinite(a).all()


def test_manufactured_dirichlet_precision_sweep():
    """N = 3 manufactured solution with Dirichlet ghosts (sources and ghost data in time), run
    to T = 2^-10 in FP64, FP32 and FP32 with the split-3xTF32 GEMM form on 4x4x2 .. 16x16x2
    meshes: each GPU state matches the oracle's (FP64 1e-10, FP32 and 3xTF32 1e-5 normwise)
    and each mode converges at order ~4 in L2."""
    from synth import manufactured_dirichlet
    from oracle.rhs import error_norms
    errs = {rdg.FP64: [], rdg.FP32: [], rdg.FP32_3XTF32: []}
    for mm in (4, 8, 16):
        w = manufactured_dirichlet(mm, N=3)
        me = Mesh(w.xy, w.tri, w.N, bc=DIRICHLET)
        osrc = [(f(me.x, me.y), k, o) for f, k, o in zip(w.source.funcs, w.source.kinds, w.source.omegas)]
        pr = Problem(me, w.D_elem, source=osrc, ghost_fn=w.exact)
        T = w.meta["T"]
        dt = stable_dt(pr, 0.5, 30)
        n = int(math.ceil(T / dt))
        dt = T / n
        want = pr.solve(w.exact(me.x, me.y, 0.0), 0.0, dt, n)
        for prec in (rdg.FP64, rdg.FP32, rdg.FP32_3XTF32):
            s = rdg.Solver(w.xy, w.tri, w.N, w.D_elem, bc=rdg.BC_DIRICHLET, period=None, precision=prec)
            xyn = s.node_coords()
            gxy = s.ghost_coords()
            s.set_forcing([(f(xyn[..., 0], xyn[..., 1]), k, o) for f, k, o in
                           zip(w.source.funcs, w.source.kinds, w.source.omegas)],
                          [(f(gxy[..., 0], gxy[..., 1]), k, o) for f, k, o in
                           zip(w.ghost.funcs, w.ghost.kinds, w.ghost.omegas)])
            s.set_state(w.exact(xyn[..., 0], xyn[..., 1], 0.0))
            s.solve_to_time(0.0, dt, n)
            got = s.get_state_host().astype(np.float64)
            s.synchronize()
            assert parity_err(got, want) < (1e-10 if prec == rdg.FP64 else 1e-5)
            errs[prec].append(error_norms(me, got, w.exact, T)[0])
            s.close()
    for prec in errs:
        order = math.log2(errs[prec][1] / errs[prec][2])
        assert 3.5 < order < 4.5, (prec, errs[prec])


@pytest.mark.parametrize("prec", [rdg.FP64, rdg.FP32])
def test_state_round_trip_through_host_tensors(prec):
    """set_state/get_state with (pinned) host tensors copy exactly what the NumPy path does."""
    s, me, D = _setup(3, prec=prec, m=5)
    u = random_nodal(s.K, s.Np, 21).astype(s.np_dtype)
    pinned = torch.from_numpy(u.copy()).pin_memory()
    s.set_state(pinned)
    out = torch.empty_like(pinned).pin_memory()
    s.get_state(out)
    assert np.array_equal(out.numpy(), u)
    assert np.array_equal(s.get_state_host(), u)
    s.close()
