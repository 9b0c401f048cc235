"""The allocation-free right-hand side (rdg_rhs_eval_static) against rdg_rhs_eval.

Some callers cannot allocate device memory where they evaluate the right-hand side (during
another component's graph capture, in loops that must not synchronise on cudaMalloc, under
a pool allocator).  rdg_rhs_eval_static keeps its per-edge fluxes in a fixed static device
array instead of a context buffer, and runs the unfused edge and element kernels rather than
the fused pair of rdg_rhs_eval.  This test calls both entry points through the C ABI on the
same input, twice in a row (the static array keeps the previous call's contents), at every
order in both precisions (FP32 order 6 included, whose rdg_rhs_eval forms the volume term on
the tensor cores), and on a Dirichlet problem with time-dependent sources and ghost data, and
checks that they agree element by element within the parity tolerance (FP32 1e-5, FP64
1e-12); it also checks the size limit and the refusal of GEMM-form contexts."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _both(lib, s, u, t):
    ref = torch.empty_like(u)
    got = torch.full_like(u, float("nan"))
    assert lib.rdg_rhs_eval(s.ctx, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(ref.data_ptr()), t) == 0
    assert lib.rdg_rhs_eval_static(s.ctx, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(got.data_ptr()), t) == 0
    torch.cuda.synchronize()
    g, r = got.double().cpu().numpy(), ref.double().cpu().numpy()
    return max(np.abs(g - r).max() / np.abs(r).max(), np.linalg.norm(g - r) / np.linalg.norm(r))


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06221_gb300 as rdg
    return rdg, rdg.load()


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_static_scratch_rhs_matches_rhs_eval(N):
    rdg, lib = _lib()
    from synth import unit_square_mesh, random_nodal
    for prec, tol in ((rdg.FP32, 1e-5), (rdg.FP64, 1e-12)):
        xy, tri = unit_square_mesh(20, 0.1, 4)
        D = np.where(np.arange(tri.shape[0]) % 5 == 0, 1.0, 0.1)
        s = rdg.Solver(xy, tri, N, D, v=(0.5, -0.25), precision=prec)
        for call, seed in enumerate((1, 2)):          # two calls in a row, different inputs
            u = torch.tensor(random_nodal(s.K, s.Np, seed), dtype=s.dtype, device="cuda")
            err = _both(lib, s, u, 0.0)
            assert err < tol, (N, prec, call, err)
        s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_static_scratch_dirichlet_with_sources(prec):
    """The manufactured Dirichlet problem (time-dependent source and ghost data) at two times."""
    rdg, lib = _lib()
    from synth import manufactured_dirichlet
    w = manufactured_dirichlet(12, N=3)
    p = rdg.FP32 if prec == "fp32" else rdg.FP64
    s = rdg.Solver(w.xy, w.tri, w.N, w.D_elem, bc=rdg.BC_DIRICHLET, period=None, precision=p)
    xyn = s.node_coords()
    gxy = s.ghost_coords()
    s.set_forcing([(f(xyn[..., 0], xyn[..., 1]), k, o) for f, k, o in zip(w.source.funcs, w.source.kinds, w.source.omegas)],
                  [(f(gxy[..., 0], gxy[..., 1]), k, o) for f, k, o in zip(w.ghost.funcs, w.ghost.kinds, w.ghost.omegas)])
    u = torch.tensor(w.exact(xyn[..., 0], xyn[..., 1], 0.3) + 0.01 * xyn[..., 0], dtype=s.dtype, device="cuda")
    for t in (0.3, 1.1):
        err = _both(lib, s, u, t)
        assert err < (1e-5 if prec == "fp32" else 1e-12), (t, err)
    s.close()


def test_static_scratch_limits():
    rdg, lib = _lib()
    from synth import unit_square_mesh, random_nodal
    # a mesh whose fluxes exceed the static array is refused with a message
    xy, tri = unit_square_mesh(230, 0.0, 0)           # 158700 edges x 7 x 8 B > 8 MiB
    s = rdg.Solver(xy, tri, 6, 1.0, precision=rdg.FP64)
    u = torch.zeros((s.K, s.Np), dtype=torch.float64, device="cuda")
    r = torch.empty_like(u)
    rc = lib.rdg_rhs_eval_static(s.ctx, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(r.data_ptr()), 0.0)
    assert rc == rdg.rdg.RDG_EINVAL
    assert b"static scratch" in lib.rdg_last_error(s.ctx)
    s.close()
    # a context with the GEMM form of the edge flux (no stored operators) is refused; the
    # same precision at order 6 keeps stored operators and is accepted
    xy, tri = unit_square_mesh(6, 0.1, 1)
    g = rdg.Solver(xy, tri, 3, 1.0, precision=rdg.FP32_3XTF32)
    u = torch.tensor(random_nodal(g.K, g.Np, 3), dtype=torch.float32, device="cuda")
    r = torch.empty_like(u)
    rc = lib.rdg_rhs_eval_static(g.ctx, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(r.data_ptr()), 0.0)
    assert rc == rdg.rdg.RDG_ESTATE and b"GEMM form" in lib.rdg_last_error(g.ctx)
    g.close()
    g6 = rdg.Solver(xy, tri, 6, 1.0, precision=rdg.FP32_3XTF32)
    u = torch.tensor(random_nodal(g6.K, g6.Np, 3), dtype=torch.float32, device="cuda")
    assert _both(lib, g6, u, 0.0) < 1e-5
    g6.close()
