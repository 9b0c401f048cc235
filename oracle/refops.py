"""Reference-element operators for the oracle (test infrastructure only).

Follows the paper's Sec. 3 (nodal DG on the reference triangle I = {r,s >= -1, r+s <= 0},
orthonormal modal basis psi_j, Vandermonde V_ij = psi_j(x_i), mass M, stiffness S, LIFT),
Sec. 4.4 (three node orderings of I so that face f is the hypotenuse, rotation
Vandermondes V_rf) and Sec. 4.5 (weak-equality reconstruction on the two halves I and
I^{-1} of the logical square with the tensor Legendre basis, Mp = (P+1)^2 unknowns,
2 Np equations, least squares).

Conventions (interface conventions shared with the CUDA library, not code):
  * vertices of I: v1 = (-1,-1), v2 = (1,-1), v3 = (-1,1);
    faces f = 1 (v1->v2), 2 (v2->v3, the hypotenuse), 3 (v3->v1), counter-clockwise.
  * nodes ordered row by row: for i = 0..N (s level), j = 0..N-i (r index).
  * face nodes listed counter-clockwise from the face's first vertex to its second.
  * "LGL nodes" on the triangle are read as the Warp & Blend construction with alpha = 0
    (LGL points on every edge).

Independent routes used here on purpose: Legendre/Jacobi values come from NumPy/SciPy
library routines with explicit normalisation, LGL points are the roots of (1-x^2) P_N'
from numpy.polynomial, differentiation matrices come from a monomial basis, and
quadrature from numpy's Gauss-Legendre rule on collapsed coordinates.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np
from numpy.polynomial import legendre as L
from scipy.special import eval_jacobi, gammaln


# ----------------------------------------------------------------------------------
# 1D
# ----------------------------------------------------------------------------------

def lgl_nodes(N: int) -> np.ndarray:
    """Legendre-Gauss-Lobatto points: -1, 1 and the roots of P_N' (ascending)."""
    if N == 1:
        return np.array([-1.0, 1.0])
    cN = np.zeros(N + 1)
    cN[N] = 1.0
    inner = np.sort(np.real(L.legroots(L.legder(cN))))
    return np.concatenate([[-1.0], inner, [1.0]])


def legendre_normalized(n: int, x):
    """Orthonormal Legendre polynomial sqrt((2n+1)/2) P_n(x) on [-1, 1]."""
    c = np.zeros(n + 1)
    c[n] = 1.0
    return math.sqrt((2 * n + 1) / 2.0) * L.legval(x, c)


def legendre_normalized_deriv(n: int, x):
    c = np.zeros(n + 1)
    c[n] = 1.0
    return math.sqrt((2 * n + 1) / 2.0) * L.legval(x, L.legder(c)) if n > 0 else np.zeros_like(np.asarray(x, float))


def jacobi_normalized(n: int, a: float, b: float, x):
    """Jacobi polynomial P_n^{(a,b)} normalised to unit norm under weight (1-x)^a (1+x)^b."""
    # h_n = 2^{a+b+1}/(2n+a+b+1) * Gamma(n+a+1) Gamma(n+b+1) / (Gamma(n+a+b+1) n!)
    logh = ((a + b + 1) * math.log(2.0) - math.log(2 * n + a + b + 1) + gammaln(n + a + 1) + gammaln(n + b + 1)
            - gammaln(n + a + b + 1) - gammaln(n + 1))
    return eval_jacobi(n, a, b, x) / math.exp(0.5 * logh)


def lagrange_1d(xn: np.ndarray, x) -> np.ndarray:
    """Lagrange basis on points xn evaluated at x: returns [len(x), len(xn)] (product formula)."""
    x = np.atleast_1d(np.asarray(x, float))
    out = np.ones((x.size, xn.size))
    for i in range(xn.size):
        for k in range(xn.size):
            if k != i:
                out[:, i] *= (x - xn[k]) / (xn[i] - xn[k])
    return out


def face_mass_1d(N: int) -> np.ndarray:
    """M1D[a, q] = int_{-1}^{1} l_a(t) l_q(t) dt on the LGL points (Gauss rule, exact)."""
    t = lgl_nodes(N)
    xq, wq = L.leggauss(N + 2)
    lq = lagrange_1d(t, xq)
    return lq.T @ (wq[:, None] * lq)


# ----------------------------------------------------------------------------------
# Triangle nodes (Warp & Blend, alpha = 0)
# ----------------------------------------------------------------------------------

def _warp_factor(N: int, rout: np.ndarray) -> np.ndarray:
    """1D warp (LGL minus equidistant positions, interpolated) divided by the edge blend
    normalisation 1 - rout^2, set to zero at the end points."""
    lgl = lgl_nodes(N)
    req = np.linspace(-1.0, 1.0, N + 1)
    warp = lagrange_1d(req, rout) @ (lgl - req)
    inside = np.abs(rout) < 1.0 - 1e-10
    sf = 1.0 - (rout * inside) ** 2
    return warp / sf + warp * (inside - 1.0)


@lru_cache(maxsize=None)
def nodes(N: int):
    """Warp & Blend nodes (alpha = 0) on I, in the row-by-row order.  Returns (r, s)."""
    L1, L3 = [], []
    for i in range(N + 1):
        for j in range(N + 1 - i):
            L1.append(i / N)
            L3.append(j / N)
    L1 = np.array(L1)
    L3 = np.array(L3)
    L2 = 1.0 - L1 - L3
    x = -L2 + L3
    y = (-L2 - L3 + 2.0 * L1) / math.sqrt(3.0)
    b1, b2, b3 = 4 * L2 * L3, 4 * L1 * L3, 4 * L1 * L2
    w1 = b1 * _warp_factor(N, L3 - L2)
    w2 = b2 * _warp_factor(N, L1 - L3)
    w3 = b3 * _warp_factor(N, L2 - L1)
    x = x + w1 + math.cos(2 * math.pi / 3) * w2 + math.cos(4 * math.pi / 3) * w3
    y = y + math.sin(2 * math.pi / 3) * w2 + math.sin(4 * math.pi / 3) * w3
    # equilateral -> reference triangle through barycentric coordinates
    l1 = (math.sqrt(3.0) * y + 1.0) / 3.0
    l2 = (-3.0 * x - math.sqrt(3.0) * y + 2.0) / 6.0
    l3 = (3.0 * x - math.sqrt(3.0) * y + 2.0) / 6.0
    r = -l2 + l3 - l1
    s = -l2 - l3 + l1
    r.setflags(write=False)
    s.setflags(write=False)
    return r, s


def num_nodes(N: int) -> int:
    return (N + 1) * (N + 2) // 2


# ----------------------------------------------------------------------------------
# Orthonormal modal basis psi on I (collapsed-coordinate Koornwinder/Dubiner)
# ----------------------------------------------------------------------------------

def mode_list(N: int):
    return [(i, j) for i in range(N + 1) for j in range(N + 1 - i)]


def psi(N: int, r, s) -> np.ndarray:
    """psi_m(r, s) for all Np modes: returns [len(r), Np].  psi_{ij} = sqrt(2) P_i(a)
    P_j^{(2i+1,0)}(b) (1-b)^i with a = 2(1+r)/(1-s) - 1, b = s."""
    r = np.atleast_1d(np.asarray(r, float))
    s = np.atleast_1d(np.asarray(s, float))
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(np.abs(s - 1.0) > 1e-14, 2.0 * (1.0 + r) / (1.0 - s) - 1.0, -1.0)
    b = s
    out = np.empty((r.size, num_nodes(N)))
    for m, (i, j) in enumerate(mode_list(N)):
        out[:, m] = math.sqrt(2.0) * jacobi_normalized(i, 0, 0, a) * jacobi_normalized(j, 2 * i + 1, 0, b) * (1 - b) ** i
    return out


def monomials(N: int, r, s):
    """Monomial basis r^p s^q (p+q <= N) and its r-, s-derivatives, each [len(r), Np]."""
    r = np.atleast_1d(np.asarray(r, float))
    s = np.atleast_1d(np.asarray(s, float))
    pq = [(p, q) for p in range(N + 1) for q in range(N + 1 - p)]
    Vm = np.stack([r ** p * s ** q for p, q in pq], axis=1)
    Vmr = np.stack([(p * r ** (p - 1) if p > 0 else 0 * r) * s ** q for p, q in pq], axis=1)
    Vms = np.stack([r ** p * (q * s ** (q - 1) if q > 0 else 0 * s) for p, q in pq], axis=1)
    return Vm, Vmr, Vms


def triangle_quadrature(deg: int):
    """Collapsed Gauss-Legendre rule on I exact for total degree <= deg.  Returns (r, s, w)."""
    q = deg // 2 + 2
    x, w = L.leggauss(q)
    A, B = np.meshgrid(x, x, indexing="ij")
    WA, WB = np.meshgrid(w, w, indexing="ij")
    r = (1 + A) * (1 - B) / 2 - 1
    s = B
    wt = WA * WB * (1 - B) / 2
    return r.ravel(), s.ravel(), wt.ravel()


# ----------------------------------------------------------------------------------
# Element operators (Sec. 3)
# ----------------------------------------------------------------------------------

class RefOps:
    """All reference-element and reconstruction operators for polynomial order N."""

    def __init__(self, N: int):
        self.N = N
        self.Np = num_nodes(N)
        self.Nfp = N + 1
        self.Mp = (N + 1) ** 2
        self.r, self.s = nodes(N)
        # Vandermonde and mass matrix with the orthonormal basis (Eq. Vandermonde)
        self.V = psi(N, self.r, self.s)
        self.Vinv = np.linalg.inv(self.V)
        self.M = np.linalg.inv(self.V @ self.V.T)
        self.Minv = np.linalg.inv(self.M)
        # differentiation matrices through the monomial basis (basis independent)
        Vm, Vmr, Vms = monomials(N, self.r, self.s)
        Vm_inv = np.linalg.inv(Vm)
        self.Dr = Vmr @ Vm_inv
        self.Ds = Vms @ Vm_inv
        # reference stiffness S_r[i,j] = int l_i d_r l_j = (M Dr)_{ij}
        self.Sr = self.M @ self.Dr
        self.Ss = self.M @ self.Ds
        # face node lists (counter-clockwise along each face)
        self.Fmask = self._face_masks()
        self.tface = lgl_nodes(N)
        # surface mass E_f (Np x Nfp) and LIFT_f = M^{-1} E_f
        M1D = face_mass_1d(N)
        self.E = np.zeros((3, self.Np, self.Nfp))
        for f in range(3):
            self.E[f][self.Fmask[f], :] = M1D
        self.LIFT = np.einsum("ij,fjq->fiq", self.Minv, self.E)
        # rotated node coordinates and Vandermondes V_rf (Sec. 4.4)
        self.rot_rs = [self.rotated_coords(f) for f in range(3)]
        self.Vr = [psi(N, *self.rot_rs[f]) for f in range(3)]
        self.Vr_inv = [np.linalg.inv(Vr) for Vr in self.Vr]
        # reconstruction system (Sec. 4.5)
        self._build_reconstruction()

    def _face_masks(self):
        N = self.N
        idx = {}
        k = 0
        for i in range(N + 1):
            for j in range(N + 1 - i):
                idx[(i, j)] = k
                k += 1
        f1 = [idx[(0, j)] for j in range(N + 1)]                 # s = -1, v1 -> v2
        f2 = [idx[(i, N - i)] for i in range(N + 1)]             # r + s = 0, v2 -> v3
        f3 = [idx[(i, 0)] for i in range(N, -1, -1)]             # r = -1, v3 -> v1
        return [np.array(f1), np.array(f2), np.array(f3)]

    def rotated_coords(self, f: int):
        """Coordinates of the nodes in the ordering of I that puts face f on the hypotenuse:
        the face's first vertex goes to (1,-1), its second to (-1,1), the opposite vertex
        to (-1,-1) (the orderings listed in Sec. 4.4)."""
        lam = np.stack([-(self.r + self.s) / 2, (self.r + 1) / 2, (self.s + 1) / 2])  # weights of v1, v2, v3
        a, b, c = [(0, 1, 2), (1, 2, 0), (2, 0, 1)][f]   # face (va, vb), apex vc
        return 2 * lam[a] - 1, 2 * lam[b] - 1

    # -- reconstruction ---------------------------------------------------------------
    def phi(self, R, S):
        """Tensor orthonormal Legendre basis phi_{ab}(R,S) = p_a(R) p_b(S), a,b = 0..N."""
        R = np.atleast_1d(R)
        S = np.atleast_1d(S)
        N = self.N
        return np.stack([legendre_normalized(a, R) * legendre_normalized(b, S)
                         for a in range(N + 1) for b in range(N + 1)], axis=1)

    def phi_grad(self, R, S):
        R = np.atleast_1d(R)
        S = np.atleast_1d(S)
        N = self.N
        dR = np.stack([legendre_normalized_deriv(a, R) * legendre_normalized(b, S)
                       for a in range(N + 1) for b in range(N + 1)], axis=1)
        dS = np.stack([legendre_normalized(a, R) * legendre_normalized_deriv(b, S)
                       for a in range(N + 1) for b in range(N + 1)], axis=1)
        return dR, dS

    def _build_reconstruction(self):
        # A1[m,n] = int_I phi_n(r,s) psi_m(r,s);  A2[m,n] = int_I phi_n(-r,-s) psi_m(r,s)
        rq, sq, wq = triangle_quadrature(3 * self.N + 2)
        P = psi(self.N, rq, sq)
        self.A1 = P.T @ (wq[:, None] * self.phi(rq, sq))
        self.A2 = P.T @ (wq[:, None] * self.phi(-rq, -sq))
        self.A = np.vstack([self.A1, self.A2])
        sv = np.linalg.svd(self.A, compute_uv=False)
        self.A_cond = sv[-1] / sv[0]
        self.Apinv = np.linalg.pinv(self.A, rcond=1e-13)
        # diagonal nodes of the parallelogram: side 1's hypotenuse nodes in its face order,
        # (R, S) = (-t, t), t ascending LGL
        t = self.tface
        self.diag_R = -t
        self.diag_S = t
        self.DR, self.DS = self.phi_grad(self.diag_R, self.diag_S)
