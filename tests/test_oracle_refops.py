"""Pins for the oracle's reference-element operators against closed forms, invariants and
independent library routines (no GPU)."""
import math
import os

import numpy as np
import pytest

from oracle.refops import (RefOps, lgl_nodes, nodes, psi, triangle_quadrature, monomials, face_mass_1d)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_lgl_closed_forms():
    # textbook closed forms of the Lobatto points
    assert np.allclose(lgl_nodes(1), [-1, 1], atol=0)
    assert np.allclose(lgl_nodes(2), [-1, 0, 1], atol=1e-15)
    a = 1 / math.sqrt(5)
    assert np.allclose(lgl_nodes(3), [-1, -a, a, 1], atol=1e-15)
    b = math.sqrt(3 / 7)
    assert np.allclose(lgl_nodes(4), [-1, -b, 0, b, 1], atol=1e-15)


def test_nodes_low_order_closed_forms():
    r, s = nodes(1)
    assert np.allclose(np.stack([r, s], 1), [[-1, -1], [1, -1], [-1, 1]], atol=1e-15)
    r, s = nodes(2)   # vertices and edge midpoints
    assert np.allclose(np.stack([r, s], 1), [[-1, -1], [0, -1], [1, -1], [-1, 0], [0, 0], [-1, 1]], atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_nodes_edges_are_lgl_and_symmetric(N):
    ops = RefOps(N)
    t = lgl_nodes(N)
    verts = np.array([[-1, -1], [1, -1], [-1, 1]], float)
    for f, (a, b) in enumerate([(0, 1), (1, 2), (2, 0)]):
        pts = np.stack([ops.r[ops.Fmask[f]], ops.s[ops.Fmask[f]]], 1)
        want = verts[a] + (t[:, None] + 1) / 2 * (verts[b] - verts[a])
        assert np.allclose(pts, want, atol=1e-14)
    # each rotated ordering is a permutation of the node set (Sec. 4.4)
    P = np.stack([ops.r, ops.s], 1)
    for f in range(3):
        R = np.stack(ops.rot_rs[f], 1)
        d = np.linalg.norm(R[:, None, :] - P[None, :, :], axis=2)
        perm = d.argmin(1)
        assert np.all(d.min(1) < 1e-13) and len(set(perm)) == ops.Np
        # V_rf = Pi_f V
        assert np.allclose(ops.Vr[f], ops.V[perm], atol=1e-13)


@pytest.mark.parametrize("N", [1, 3, 6])
def test_psi_orthonormal(N):
    rq, sq, wq = triangle_quadrature(2 * N)
    P = psi(N, rq, sq)
    G = P.T @ (wq[:, None] * P)
    assert np.allclose(G, np.eye(P.shape[1]), atol=1e-12)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_mass_and_derivatives(N):
    ops = RefOps(N)
    assert abs(ops.M.sum() - 2.0) < 1e-13              # |I| = 2
    # M_ij = int l_i l_j by quadrature of the Lagrange basis built from monomials
    rq, sq, wq = triangle_quadrature(2 * N)
    Vm, _, _ = monomials(N, ops.r, ops.s)
    Vq, _, _ = monomials(N, rq, sq)
    lag = Vq @ np.linalg.inv(Vm)
    assert np.allclose(lag.T @ (wq[:, None] * lag), ops.M, atol=1e-12)
    # derivatives of all monomials of degree <= N are exact
    rng = np.random.default_rng(N)
    for p in range(N + 1):
        for q in range(N + 1 - p):
            u = ops.r ** p * ops.s ** q
            ur = p * ops.r ** max(p - 1, 0) * ops.s ** q if p else 0 * u
            us = q * ops.r ** p * ops.s ** max(q - 1, 0) if q else 0 * u
            assert np.allclose(ops.Dr @ u, ur, atol=1e-10 * (1 + np.abs(ur).max()))
            assert np.allclose(ops.Ds @ u, us, atol=1e-10 * (1 + np.abs(us).max()))


@pytest.mark.parametrize("N", [1, 2, 4, 6])
def test_lift_integrates_face_values(N):
    """M LIFT_f u|_f = int_f l_i u dt for polynomial traces (degree-2N Gauss rule)."""
    ops = RefOps(N)
    rng = np.random.default_rng(7)
    co = rng.standard_normal(N + 1)
    xg, wg = np.polynomial.legendre.leggauss(N + 2)
    verts = np.array([[-1, -1], [1, -1], [-1, 1]], float)
    Vm, _, _ = monomials(N, ops.r, ops.s)
    for f, (a, b) in enumerate([(0, 1), (1, 2), (2, 0)]):
        trace = np.polyval(co, ops.tface)
        lhs = ops.M @ (ops.LIFT[f] @ trace)
        pts = verts[a] + (xg[:, None] + 1) / 2 * (verts[b] - verts[a])
        Vq, _, _ = monomials(N, pts[:, 0], pts[:, 1])
        lag = Vq @ np.linalg.inv(Vm)
        rhs = lag.T @ (wg * np.polyval(co, xg))
        assert np.allclose(lhs, rhs, atol=1e-12)


def test_face_mass_1d_closed_form():
    # N = 1: linear Lagrange on [-1, 1]: [[2/3, 1/3], [1/3, 2/3]]
    assert np.allclose(face_mass_1d(1), [[2 / 3, 1 / 3], [1 / 3, 2 / 3]], atol=1e-15)


def test_parallelogram_storage_table():
    """Mp = (P+1)^2 tensor modes and Mp^2 reference mass entries (Table ardg_storage)."""
    rows = [list(map(int, l.split())) for l in open(os.path.join(GOLDEN, "ardg_storage.txt")) if l[0] != "#"]
    for P, NP, J, RX, Msz in rows:
        ops = RefOps(P)
        assert ops.Mp == NP and ops.A.shape == (2 * ops.Np, NP)
        assert NP * NP == Msz and J == 1 and RX == 4


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_reconstruction_system_rank_and_exactness(N):
    ops = RefOps(N)
    assert ops.A_cond > 1e-10
    # a global degree-N polynomial written in the tensor basis is reproduced exactly:
    # its weak moments on I and I^{-1} equal the projections of the same polynomial
    rng = np.random.default_rng(N)
    co = {(a, b): rng.standard_normal() for a in range(N + 1) for b in range(N + 1 - a)}
    p = lambda R, S: sum(c * R ** a * S ** b for (a, b), c in co.items())
    # tensor coefficients of p by least squares on a fine grid
    g = np.linspace(-1, 1, 3 * N + 3)
    Rg, Sg = [x.ravel() for x in np.meshgrid(g, g)]
    cten = np.linalg.lstsq(ops.phi(Rg, Sg), p(Rg, Sg), rcond=None)[0]
    rq, sq, wq = triangle_quadrature(2 * N)
    P = psi(N, rq, sq)
    m1 = P.T @ (wq * p(rq, sq))
    m2 = P.T @ (wq * p(-rq, -sq))
    assert np.allclose(ops.A @ cten, np.concatenate([m1, m2]), atol=1e-11)
    assert np.allclose(ops.Apinv @ np.concatenate([m1, m2]), cten, atol=1e-10)
