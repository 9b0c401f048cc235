"""Pins for the oracle's enclosed parallelogram, projections and reconstruction (no GPU)."""
import numpy as np
import pytest

from synth import unit_square_mesh, PERIODIC, DIRICHLET
from oracle.mesh import Mesh, FACE_APEX, FACE_VERTS
from oracle.ardg import EdgeOps, enclosed_parallelogram
from oracle.rhs import Problem


def _bary(p, a, b, c):
    T = np.column_stack([b - a, c - a])
    l = np.linalg.solve(T, p - a)
    return np.array([1 - l.sum(), l[0], l[1]])


def _poly(N, seed):
    rng = np.random.default_rng(seed)
    co = {(a, b): rng.standard_normal() for a in range(N + 1) for b in range(N + 1 - a)}
    f = lambda x, y: sum(c * x ** a * y ** b for (a, b), c in co.items())
    fx = lambda x, y: sum(c * a * x ** (a - 1) * y ** b for (a, b), c in co.items() if a)
    fy = lambda x, y: sum(c * b * x ** a * y ** (b - 1) for (a, b), c in co.items() if b)
    return f, fx, fy


def test_parallelogram_on_unjittered_mesh_is_the_quad():
    xy, tri = unit_square_mesh(4, 0.0)
    m = Mesh(xy, tri, 2)
    eo = EdgeOps(m)
    for e, (k1, f1, k2, f2, sx, sy) in enumerate(m.edges):
        q1 = m.V[k1, FACE_APEX[f1]]
        q2 = m.V[k2, FACE_APEX[f2]] + [sx, sy]
        assert np.allclose(eo.p1[e], q1, atol=1e-14) and np.allclose(eo.p2[e], q2, atol=1e-14)
        # apexes of the sub-triangles sit at the reference apex in each rotated frame
        assert np.allclose(eo.ab1[e], [-1, -1], atol=1e-13) and np.allclose(eo.ab2[e], [-1, -1], atol=1e-13)


def test_parallelogram_brute_force_and_containment():
    rng = np.random.default_rng(11)
    for trial in range(60):
        e1 = np.array([0.0, 0.0]) + rng.uniform(-0.2, 0.2, 2)
        e2 = np.array([1.0, 0.0]) + rng.uniform(-0.2, 0.2, 2)
        q1 = np.array([rng.uniform(-0.5, 1.5), rng.uniform(0.2, 1.5)])
        q2 = np.array([rng.uniform(-0.5, 1.5), rng.uniform(-1.5, -0.2)])
        p1, p2 = enclosed_parallelogram(e1, e2, q1, q2)
        c = (e1 + e2) / 2
        assert np.allclose(p1 + p2, 2 * c, atol=1e-13)
        assert _bary(p1, e1, e2, q1).min() > -1e-12
        assert _bary(p2, e2, e1, q2).min() > -1e-12
        d = e2 - e1
        height = lambda p: d[0] * (p[1] - e1[1]) - d[1] * (p[0] - e1[0])
        # area of the parallelogram <= twice the area of either triangle
        assert height(p1) <= height(q1) + 1e-12 and height(p1) <= -height(q2) + 1e-12
        # brute force: no point of T1 whose reflection lies in T2 is higher than p1
        w = rng.dirichlet([1, 1, 1], 4000)
        pts = w[:, 0:1] * e1 + w[:, 1:2] * e2 + w[:, 2:3] * q1
        refl = 2 * c - pts
        ok = np.array([_bary(r, e2, e1, q2).min() >= 0 for r in refl])
        hs = np.array([height(p) for p in pts[ok]])
        assert hs.size == 0 or hs.max() <= height(p1) + 1e-12
        # vertex enumeration (an independent route): the highest point of T1 n T2' is a
        # vertex of one triangle or a crossing of two edge lines lying in both triangles
        T1 = [e1, e2, q1]
        T2r = [e1, e2, 2 * c - q2]
        cand = list(T1) + list(T2r)
        for i in range(3):
            for j in range(3):
                a0, a1 = T1[i], T1[(i + 1) % 3]
                b0, b1 = T2r[j], T2r[(j + 1) % 3]
                Mx = np.column_stack([a1 - a0, b0 - b1])
                if abs(np.linalg.det(Mx)) > 1e-14:
                    st = np.linalg.solve(Mx, b0 - a0)
                    cand.append(a0 + st[0] * (a1 - a0))
        inside = [p for p in cand if _bary(p, e1, e2, q1).min() > -1e-12 and _bary(p, e1, e2, 2 * c - q2).min() > -1e-12]
        assert abs(max(height(p) for p in inside) - height(p1)) < 1e-12
        # swapping the two sides gives the same parallelogram
        p1s, p2s = enclosed_parallelogram(e2, e1, q2, q1)
        assert np.allclose(p1s, p2, atol=1e-12) and np.allclose(p2s, p1, atol=1e-12)


def test_parallelogram_special_cases():
    e1, e2 = np.array([0.0, 0.0]), np.array([2.0, 0.0])
    # reflected apex of T2 inside T1: p1 is that reflected apex
    q1, q2 = np.array([1.0, 2.0]), np.array([1.0, -1.0])
    p1, _ = enclosed_parallelogram(e1, e2, q1, q2)
    assert np.allclose(p1, [1.0, 1.0])
    # both apexes at the same height but shifted: crossing of the two slanted edges
    q1, q2 = np.array([0.0, 1.0]), np.array([0.0, -1.0])   # 2c - q2 = (2, 1)
    p1, _ = enclosed_parallelogram(e1, e2, q1, q2)
    assert np.allclose(p1, [1.0, 0.5])


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("bc", [PERIODIC, DIRICHLET])
def test_reconstruction_reproduces_global_polynomials(N, bc):
    """If u1, u2 restrict one polynomial p of degree <= N, u~ = p and g = n.grad p."""
    xy, tri = unit_square_mesh(4, 0.1, 3)
    m = Mesh(xy, tri, N, bc=bc)
    f, fx, fy = _poly(N, N + 10 * bc)
    pr = Problem(m, np.ones(m.K), ghost_fn=lambda x, y, t: f(x, y))
    u = f(m.x, m.y)
    ops = m.ops
    wrapped = np.array([abs(e[4]) + abs(e[5]) > 1e-12 for e in m.edges])
    u2 = np.zeros((m.E, ops.Np))
    u2[pr.interior] = u[pr.k2[pr.interior]]
    if pr.bnd.size:
        u2[pr.bnd] = pr.ghost_values(0.0)
    c = pr.eops.reconstruct(u[pr.k1], u2)
    g = pr.eops.edge_normal_gradient(c)
    fxn = np.stack([m.x[k, ops.Fmask[ff]] for k, ff in zip(pr.k1, pr.f1)])
    fyn = np.stack([m.y[k, ops.Fmask[ff]] for k, ff in zip(pr.k1, pr.f1)])
    n1 = pr.eops.n1
    gex = n1[:, :1] * fx(fxn, fyn) + n1[:, 1:] * fy(fxn, fyn)
    assert np.abs(g - gex)[~wrapped].max() < 1e-10 * (1 + np.abs(gex).max())
    uval = pr.eops.reconstructed_values(c)
    assert np.abs(uval - f(fxn, fyn))[~wrapped].max() < 1e-11


@pytest.mark.parametrize("N", [2, 4])
def test_reconstruction_swap_invariance(N):
    """Taking the other element as side 1 negates and reverses the edge gradient."""
    xy, tri = unit_square_mesh(4, 0.1, 9)
    m = Mesh(xy, tri, N)
    eo = EdgeOps(m)
    rng = np.random.default_rng(0)
    u = rng.standard_normal((m.K, m.ops.Np))
    k1 = np.array([e[0] for e in m.edges])
    k2 = np.array([e[2] for e in m.edges])
    g = eo.edge_normal_gradient(eo.reconstruct(u[k1], u[k2]))
    m.edges = [(k2_, f2, k1_, f1, -sx, -sy) for (k1_, f1, k2_, f2, sx, sy) in m.edges]
    eo2 = EdgeOps(m)
    g2 = eo2.edge_normal_gradient(eo2.reconstruct(u[k2], u[k1]))
    assert np.allclose(g2, -g[:, ::-1], atol=1e-10 * np.abs(g).max())


@pytest.mark.parametrize("N", [1, 3, 6])
def test_algorithm2_D_is_edge_mean(N):
    """For element-constant D, RDG(D1, D2) on the diagonal equals (D1 + D2)/2 (symmetry)."""
    xy, tri = unit_square_mesh(4, 0.1, 2)
    m = Mesh(xy, tri, N)
    D = np.random.default_rng(N).uniform(1e-4, 1.0, m.K)
    pr = Problem(m, D)
    want = 0.5 * (D[pr.k1] + D[pr.k2])
    assert np.allclose(pr.Dt, want[:, None], atol=1e-12)
