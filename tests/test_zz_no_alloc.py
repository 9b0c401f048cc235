"""The allocation-free right-hand side (rdg_rhs_eval_static) against rdg_rhs_eval.

Some callers cannot allocate device memory where they evaluate the right-hand side (during
another component's graph capture, in loops that must not synchronise on cudaMalloc, under
a pool allocator).  rdg_rhs_eval_static keeps its per-edge fluxes in a fixed static device
array instead of a context buffer.  This test calls both entry points through the C ABI on
the same input, twice in a row (the static array keeps the previous call's contents), and
checks that they agree within the FP32 parity tolerance; it also checks the size limit."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_static_scratch_rhs_matches_rhs_eval():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06221_gb300 as rdg
    from synth import unit_square_mesh, random_nodal
    lib = rdg.load()
    for prec, tol in ((rdg.FP32, 1e-5), (rdg.FP64, 1e-12)):
        xy, tri = unit_square_mesh(20, 0.1, 4)
        D = np.where(np.arange(tri.shape[0]) % 5 == 0, 1.0, 0.1)
        s = rdg.Solver(xy, tri, 4, D, v=(0.5, -0.25), precision=prec)
        for call, seed in enumerate((1, 2)):          # two calls in a row, different inputs
            u = torch.tensor(random_nodal(s.K, s.Np, seed), dtype=s.dtype, device="cuda")
            ref = torch.empty_like(u)
            got = torch.full_like(u, float("nan"))
            assert lib.rdg_rhs_eval(s.ctx, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(ref.data_ptr()), 0.0) == 0
            assert lib.rdg_rhs_eval_static(s.ctx, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(got.data_ptr()),
                                           0.0) == 0
            torch.cuda.synchronize()
            err = float(torch.linalg.vector_norm(got.double() - ref.double()) / torch.linalg.vector_norm(ref.double()))
            assert err < tol, (prec, call, err)
        s.close()
    # a mesh whose fluxes exceed the static array is refused with a message
    xy, tri = unit_square_mesh(230, 0.0, 0)           # 158700 edges x 7 x 8 B > 8 MiB
    s = rdg.Solver(xy, tri, 6, 1.0, precision=rdg.FP64)
    u = torch.zeros((s.K, s.Np), dtype=torch.float64, device="cuda")
    r = torch.empty_like(u)
    rc = lib.rdg_rhs_eval_static(s.ctx, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(r.data_ptr()), 0.0)
    assert rc == rdg.rdg.RDG_EINVAL
    assert b"static scratch" in lib.rdg_last_error(s.ctx)
    s.close()
