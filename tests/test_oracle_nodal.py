"""Pins for the oracle's spatially varying (nodal) D (Sec. 3: D a function of space in Eq.
NDG_diffusion_once_matrixForm_reference_general; Algorithms 1 and 2 applied to it).

* Exactness: D linear in space and p a global polynomial of degree <= N - 1: D grad p has
  degree <= N, so the nodal product, the reconstruction of D (Algorithm 2), the projection of
  D onto the sub-triangles (Algorithm 1) and the traces (harmonic rule) are all exact, and the
  right-hand side is div(D grad p) - v . grad p at the nodes of every element whose edges are
  not wrapped.
* A nodal D that is constant on every element gives the element-wise-D operator.
* The interface flux stays single valued: discrete conservation on a periodic mesh with a
  random positive nodal D, discontinuous across elements.
"""
import numpy as np
import pytest

from synth import unit_square_mesh, DIRICHLET
from oracle.mesh import Mesh
from oracle.rhs import Problem

IFACES = ["alg1", "alg2", "harmonic"]


def _poly(N, seed):
    rng = np.random.default_rng(seed)
    co = {(a, b): rng.standard_normal() for a in range(N + 1) for b in range(N + 1 - a)}
    f = lambda x, y: sum(c * x ** a * y ** b for (a, b), c in co.items()) + 0 * x
    fx = lambda x, y: sum(c * a * x ** (a - 1) * y ** b for (a, b), c in co.items() if a) + 0 * x
    fy = lambda x, y: sum(c * b * x ** a * y ** (b - 1) for (a, b), c in co.items() if b) + 0 * x
    lap = lambda x, y: (sum(c * a * (a - 1) * x ** (a - 2) * y ** b for (a, b), c in co.items() if a > 1)
                        + sum(c * b * (b - 1) * x ** a * y ** (b - 2) for (a, b), c in co.items() if b > 1) + 0 * x)
    return f, fx, fy, lap


def _unwrapped(m):
    good = np.ones(m.K, bool)
    for (k1, f1, k2, f2, sx, sy) in m.edges:
        if abs(sx) + abs(sy) > 1e-12:
            good[k1] = good[k2] = False
    return good


@pytest.mark.parametrize("iface", IFACES)
@pytest.mark.parametrize("N", [2, 3, 4, 6])
def test_nodal_D_exact_for_linear_D_and_polynomials(N, iface):
    xy, tri = unit_square_mesh(5, 0.1, 4)
    m = Mesh(xy, tri, N)
    a0, ax, ay = 0.5, 0.3, -0.2
    D = a0 + ax * m.x + ay * m.y
    v = (0.8, -0.45)
    pr = Problem(m, D, v=v, interface=iface)
    f, fx, fy, lap = _poly(N - 1, 300 + N)
    r = pr.rhs(f(m.x, m.y))
    X, Y = m.x, m.y
    want = D * lap(X, Y) + ax * fx(X, Y) + ay * fy(X, Y) - v[0] * fx(X, Y) - v[1] * fy(X, Y)
    good = _unwrapped(m)
    scale = 1 + np.abs(want).max()
    assert np.abs(r - want)[good].max() < 1e-9 * scale * (N + 1) ** 4


@pytest.mark.parametrize("iface", IFACES)
def test_elementwise_constant_nodal_D_equals_element_D(iface):
    for bc in (0, DIRICHLET):
        xy, tri = unit_square_mesh(5, 0.1, 7)
        m = Mesh(xy, tri, 3, bc=bc)
        d = np.random.default_rng(2).uniform(0.1, 1.0, m.K)
        g = (lambda x, y, t: 0.3 * x - y) if bc == DIRICHLET else None
        a = Problem(m, d, v=(0.3, 0.2), interface=iface, ghost_fn=g)
        b = Problem(m, np.repeat(d[:, None], m.ops.Np, axis=1), v=(0.3, 0.2), interface=iface, ghost_fn=g)
        u = np.random.default_rng(3).standard_normal((m.K, m.ops.Np))
        ra, rb = a.rhs(u, 0.1), b.rhs(u, 0.1)
        assert np.abs(ra - rb).max() < 1e-12 * np.abs(ra).max(), bc


@pytest.mark.parametrize("iface", IFACES)
def test_nodal_D_conservation(iface):
    xy, tri = unit_square_mesh(5, 0.1, 8)
    m = Mesh(xy, tri, 4)
    rng = np.random.default_rng(4)
    D = rng.uniform(0.05, 1.0, (m.K, m.ops.Np))
    pr = Problem(m, D, v=(0.4, 0.9), interface=iface)
    w = m.J[:, None] * (pr.rhs(rng.standard_normal((m.K, m.ops.Np))) @ m.ops.M)
    assert abs(w.sum()) < 1e-12 * np.abs(w).sum()
