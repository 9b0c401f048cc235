"""The C-ABI library builds, loads and exports every symbol include/rdg.h declares (no GPU:
no compute call is made)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06221_gb300 as rdg
    return rdg.load()


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rdg_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s


def test_binding_declares_every_symbol():
    from paper_1912_06221_gb300.rdg import SIGNATURES
    assert declared_symbols() == set(SIGNATURES)


def test_host_only_entry_points(lib):
    import paper_1912_06221_gb300 as rdg
    assert lib.rdg_version().startswith(b"rdg-gb300")
    # admission bytes: W operator + indices + coefficients + fluxes + state buffers
    N, K, E = 4, 131072, 196608
    b = rdg.query_bytes(N, K, E, 0, rdg.FP32)
    W = ((E + 31) // 32) * 37 * 32 * 16          # ceil((5 * 29 + 1) / 4) = 37 words per edge
    assert b == W + 12 * E + 12 * K + 3 * K * 5 * 4 + 24 * K + E * 5 * 4 + 4 * K * 15 * 4
    assert rdg.query_bytes(N, K, E, 0, rdg.FP64) > b
    with pytest.raises(rdg.RdgError):
        rdg.query_bytes(7, K, E, 0, rdg.FP32)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_library_reference_operators_match_oracle(lib, N):
    """The library's host FP64 reference operators (its own implementation) agree with the
    oracle's to rounding."""
    import paper_1912_06221_gb300 as rdg
    from oracle.refops import RefOps
    o = RefOps(N)
    rs = rdg.reference_operator(N, 0)
    assert np.abs(rs[0] - o.r).max() < 1e-14 and np.abs(rs[1] - o.s).max() < 1e-14
    sc = (N + 1) ** 2
    assert np.abs(rdg.reference_operator(N, 1) - o.Dr).max() < 1e-11 * sc
    assert np.abs(rdg.reference_operator(N, 2) - o.Ds).max() < 1e-11 * sc
    assert np.abs(rdg.reference_operator(N, 3) - np.concatenate(list(o.LIFT), axis=1)).max() < 1e-12 * sc
    assert np.abs(rdg.reference_operator(N, 4) - o.Apinv).max() < 1e-12 * sc
    assert np.abs(rdg.reference_operator(N, 5) - o.M).max() < 1e-14 * sc


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    ctx = ctypes.c_void_p()
    rc = lib.rdg_create(ctypes.byref(ctx), 0, None)
    assert rc != 0 and lib.rdg_last_error(None)


def test_missing_library_raises(tmp_path, monkeypatch):
    """No CPU fallback: without the built library every entry raises."""
    import paper_1912_06221_gb300.rdg as r
    monkeypatch.setattr(r, "_lib", None)
    with pytest.raises(RuntimeError):
        r.load(str(tmp_path / "librdg.so"))


def test_solver_without_gpu_raises(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_1912_06221_gb300 as rdg
    from synth import unit_square_mesh
    xy, tri = unit_square_mesh(4, 0.1, 1)
    with pytest.raises(Exception):
        rdg.Solver(xy, tri, 2, 1.0)


@pytest.mark.parametrize("N", [1, 2, 4, 6])
def test_library_nodal_D_factors_match_oracle(lib, N):
    """The factors of a nodal D (RVV = Phi_diag A+_j Vinv, GR/GS = D V A_j A+_k Vinv), which do
    not depend on the choice of orthonormal bases, equal the oracle's compositions, and
    s_j RVV_j GR_jk summed with unit D gives back Algorithm 1's factor for constant D."""
    import paper_1912_06221_gb300 as rdg
    from oracle.refops import RefOps
    o = RefOps(N)
    Np = o.Np
    Phi = o.phi(o.diag_R, o.diag_S)
    A = [o.A1, o.A2]
    Ap = [o.Apinv[:, :Np], o.Apinv[:, Np:]]
    RVV = rdg.reference_operator(N, 9)
    GR = rdg.reference_operator(N, 10)
    GS = rdg.reference_operator(N, 11)
    sc = (N + 1) ** 4
    for j in range(2):
        assert np.abs(RVV[j] - Phi @ Ap[j] @ o.Vinv).max() < 1e-11 * sc
        for k in range(2):
            assert np.abs(GR[j, k] - o.Dr @ o.V @ A[j] @ Ap[k] @ o.Vinv).max() < 1e-10 * sc
            assert np.abs(GS[j, k] - o.Ds @ o.V @ A[j] @ Ap[k] @ o.Vinv).max() < 1e-10 * sc
