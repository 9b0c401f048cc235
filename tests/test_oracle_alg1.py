"""Pins of the oracle's Algorithm 1 (Sec. 3: n . RDG(D_p^1 grad u~^1, D_p^2 grad u~^2), with
Separation read as the L2 projection onto each sub-triangle) against what the mathematics
fixes:

* constant D and data from one global polynomial of degree <= N: every step is exact (the
  reconstruction reproduces P_N, the projections keep it, grad p is in P_{N-1}), so the
  flux is D n . grad p at the diagonal nodes and the right-hand side is D lap p - v.grad p;
* linear data with D1 != D2: the product field is D_k g with a constant g on each side, and
  the reconstruction of that step evaluated on the diagonal is (D1 + D2)/2 g (the symmetry
  argument that gives Algorithm 2's D~), so Algorithm 1 and Algorithm 2 give the same flux;
* the flux is single valued, so the periodic right-hand side conserves the total;
* a constant state is steady for any element-wise D.
"""
import numpy as np
import pytest

from synth import unit_square_mesh
from oracle.mesh import Mesh
from oracle.rhs import Problem

from tests.test_oracle_rhs import _poly, _unwrapped_elements


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_alg1_exact_for_global_polynomials(N):
    xy, tri = unit_square_mesh(5, 0.1, 4)
    m = Mesh(xy, tri, N)
    D, v = 0.37, (0.8, -0.45)
    pr = Problem(m, np.full(m.K, D), v=v, interface="alg1")
    f, fx, fy, lap = _poly(N, 200 + N)
    u = f(m.x, m.y)
    # the edge flux itself: D n1 . grad p at side 1's face nodes
    eo = pr.eops
    u1 = u[pr.k1]
    u2 = u[np.maximum(pr.k2, 0)]
    c = eo.reconstruct(u1, u2)
    g = eo.flux_algorithm1(c, pr.D1e, pr.D2e)
    ops = m.ops
    for e in range(m.E):
        k1, f1 = pr.k1[e], pr.f1[e]
        if abs(m.edges[e][4]) + abs(m.edges[e][5]) > 1e-12:
            continue                      # wrapped edge: the data is not one polynomial there
        nodes = ops.Fmask[f1]
        want = D * (eo.n1[e, 0] * fx(m.x[k1, nodes], m.y[k1, nodes]) + eo.n1[e, 1] * fy(m.x[k1, nodes], m.y[k1, nodes]))
        assert np.abs(g[e] - want).max() < 1e-9 * (1 + np.abs(want).max()) * (N + 1) ** 2
    r = pr.rhs(u)
    want = D * lap(m.x, m.y) - v[0] * fx(m.x, m.y) - v[1] * fy(m.x, m.y)
    good = _unwrapped_elements(m)
    assert np.abs(r - want)[good].max() < 1e-9 * (1 + np.abs(want).max()) * (N + 1) ** 4


@pytest.mark.parametrize("N", [1, 2, 4, 6])
def test_alg1_equals_alg2_for_linear_data(N):
    xy, tri = unit_square_mesh(5, 0.1, 6)
    m = Mesh(xy, tri, N)
    D = np.random.default_rng(3).uniform(1e-3, 1.0, m.K)
    lin = 0.3 + 1.7 * m.x - 0.9 * m.y
    a = Problem(m, D, interface="alg1")
    b = Problem(m, D, interface="alg2")
    good = _unwrapped_elements(m)
    fa = a.edge_flux(lin)
    fb = b.edge_flux(lin)
    inner = np.array([abs(e[4]) + abs(e[5]) < 1e-12 for e in m.edges])
    assert np.abs(fa - fb)[inner].max() < 1e-10 * np.abs(fb).max()
    assert np.abs(a.rhs(lin) - b.rhs(lin))[good].max() < 1e-9 * (N + 1) ** 4 * 25


@pytest.mark.parametrize("N", [1, 3, 5])
def test_alg1_conservation_and_constants(N):
    xy, tri = unit_square_mesh(5, 0.1, 8)
    m = Mesh(xy, tri, N)
    D = np.random.default_rng(1).uniform(1e-3, 1, m.K)
    pr = Problem(m, D, v=(0.4, 0.9), interface="alg1")
    u = np.random.default_rng(2).standard_normal((m.K, m.ops.Np))
    r = pr.rhs(u)
    w = m.J[:, None] * (r @ m.ops.M)
    assert abs(w.sum()) < 1e-12 * np.abs(w).sum()
    assert np.abs(pr.rhs(np.full((m.K, m.ops.Np), 2.5))).max() < 1e-13 * (N + 1) ** 4 * 75


def test_alg1_differs_from_alg2_only_by_truncation():
    """The two readings are different operators (not a relabelling), and on smooth data with
    constant D they differ only by the truncation of the projected gradient: the relative
    difference of the right-hand sides shrinks under refinement (the paper reports minimal
    differences between the two formulations)."""
    d = []
    for msz in (4, 8):
        xy, tri = unit_square_mesh(msz, 0.1, 2)
        m = Mesh(xy, tri, 3)
        u = np.sin(2 * np.pi * m.x) * np.cos(2 * np.pi * m.y)
        a = Problem(m, np.full(m.K, 0.4), interface="alg1").rhs(u)
        b = Problem(m, np.full(m.K, 0.4), interface="alg2").rhs(u)
        d.append(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert d[0] > 1e-10 and d[1] < d[0] / 2, d
