"""Pins for the oracle's diagonal diffusion tensor D = (Dx, Dy) (Eq.
NDG_diffusion_once_matrixForm_reference_general, Sec. 3), every interface rule.

* Exactness: for a global polynomial p of degree <= N and a constant tensor, the right-hand
  side is Dx p_xx + Dy p_yy - v . grad p on every element whose edges are not wrapped (the
  reconstruction reproduces p, each sub-triangle's product D grad p is reproduced, Sec. 2.3).
* Linear data with v = 0 and constants give zero; the interface flux is single valued, so the
  discrete mass is conserved on a periodic mesh for any element-wise tensor.
* Rotating the mesh by 90 degrees swaps the roles of x and y: the rotated problem with
  (Dy, Dx) and the rotated velocity has the same right-hand side node by node (a transposed
  or swapped component fails this).
* The mode sin(2 pi x) sin(2 pi y) decays at the rate 4 pi^2 (Dx + Dy) of the exact solution.
"""
import math

import numpy as np
import pytest

from synth import unit_square_mesh
from oracle.mesh import Mesh
from oracle.rhs import Problem

IFACES = ["alg1", "alg2", "harmonic"]


def _poly(N, seed):
    rng = np.random.default_rng(seed)
    co = {(a, b): rng.standard_normal() for a in range(N + 1) for b in range(N + 1 - a)}
    f = lambda x, y: sum(c * x ** a * y ** b for (a, b), c in co.items()) + 0 * x
    fx = lambda x, y: sum(c * a * x ** (a - 1) * y ** b for (a, b), c in co.items() if a) + 0 * x
    fy = lambda x, y: sum(c * b * x ** a * y ** (b - 1) for (a, b), c in co.items() if b) + 0 * x
    fxx = lambda x, y: sum(c * a * (a - 1) * x ** (a - 2) * y ** b for (a, b), c in co.items() if a > 1) + 0 * x
    fyy = lambda x, y: sum(c * b * (b - 1) * x ** a * y ** (b - 2) for (a, b), c in co.items() if b > 1) + 0 * x
    return f, fx, fy, fxx, fyy


def _unwrapped(m):
    good = np.ones(m.K, bool)
    for (k1, f1, k2, f2, sx, sy) in m.edges:
        if abs(sx) + abs(sy) > 1e-12:
            good[k1] = good[k2] = False
    return good


@pytest.mark.parametrize("iface", IFACES)
@pytest.mark.parametrize("N", [1, 2, 3, 4, 6])
def test_tensor_rhs_exact_for_global_polynomials(N, iface):
    xy, tri = unit_square_mesh(5, 0.1, 4)
    m = Mesh(xy, tri, N)
    Dx, Dy, v = 0.9, 0.15, (0.8, -0.45)
    pr = Problem(m, np.tile([Dx, Dy], (m.K, 1)), v=v, interface=iface)
    f, fx, fy, fxx, fyy = _poly(N, 200 + N)
    r = pr.rhs(f(m.x, m.y))
    want = Dx * fxx(m.x, m.y) + Dy * fyy(m.x, m.y) - v[0] * fx(m.x, m.y) - v[1] * fy(m.x, m.y)
    good = _unwrapped(m)
    scale = 1 + np.abs(want).max()
    assert np.abs(r - want)[good].max() < 1e-9 * scale * (N + 1) ** 4


@pytest.mark.parametrize("iface", IFACES)
def test_tensor_linear_constant_and_conservation(iface):
    N = 3
    xy, tri = unit_square_mesh(5, 0.1, 6)
    m = Mesh(xy, tri, N)
    good = _unwrapped(m)
    tol = 1e-13 * (N + 1) ** 4 * 25 * 3
    rng = np.random.default_rng(3)
    D = rng.uniform(0.05, 1.0, (m.K, 2))
    pr0 = Problem(m, np.tile([0.6, 0.2], (m.K, 1)), interface=iface)
    assert np.abs(pr0.rhs(0.3 + 1.7 * m.x - 0.9 * m.y))[good].max() < tol
    pr = Problem(m, D, v=(0.2, 0.7), interface=iface)
    assert np.abs(pr.rhs(np.full((m.K, m.ops.Np), 2.5))).max() < tol
    u = rng.standard_normal((m.K, m.ops.Np))
    w = m.J[:, None] * (pr.rhs(u) @ m.ops.M)
    assert abs(w.sum()) < 1e-12 * np.abs(w).sum()


@pytest.mark.parametrize("iface", IFACES)
def test_tensor_rotation_swaps_components(iface):
    """(x, y) -> (1 - y, x) maps the periodic unit square onto itself and keeps every triangle
    counter-clockwise with the same vertex order, so nodal arrays correspond row by row."""
    N = 3
    xy, tri = unit_square_mesh(6, 0.12, 2)
    rng = np.random.default_rng(5)
    D = rng.uniform(0.05, 1.0, (tri.shape[0], 2))
    v = (0.7, -0.3)
    u = rng.standard_normal((tri.shape[0], 10))
    pr = Problem(Mesh(xy, tri, N), D, v=v, interface=iface)
    xr = np.stack([1.0 - xy[:, 1], xy[:, 0]], axis=1)
    prr = Problem(Mesh(xr, tri, N), D[:, ::-1], v=(-v[1], v[0]), interface=iface)
    a, b = pr.rhs(u), prr.rhs(u)
    assert np.abs(a - b).max() < 1e-11 * np.abs(a).max()
    # and it is not symmetric under the swap alone (the pin can fail)
    prs = Problem(Mesh(xy, tri, N), D[:, ::-1], v=v, interface=iface)
    assert np.abs(prs.rhs(u) - a).max() > 1e-3 * np.abs(a).max()


@pytest.mark.parametrize("iface", ["alg1", "alg2"])
def test_tensor_sin_mode_decay_rate(iface):
    N, m_ = 3, 12
    xy, tri = unit_square_mesh(m_, 0.1, 0)
    m = Mesh(xy, tri, N)
    Dx, Dy = 1.0, 0.25
    pr = Problem(m, np.tile([Dx, Dy], (m.K, 1)), interface=iface)
    u0 = np.sin(2 * np.pi * m.x) * np.sin(2 * np.pi * m.y)
    h = 1.0 / m_
    dt = 0.05 * h * h / ((Dx + Dy) * (N + 1) ** 2)
    n = 40
    u = pr.solve(u0, 0.0, dt, n)
    Mw = m.J[:, None] * (u0 @ m.ops.M)
    rate = math.log(np.sum(Mw * u) / np.sum(Mw * u0)) / (-4 * math.pi ** 2 * (Dx + Dy) * n * dt)
    assert abs(rate - 1) < 1e-2
