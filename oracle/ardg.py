"""Affine reconstruction on the enclosed parallelogram (Sec. 4 and Algorithm aRDG), oracle
version (test infrastructure only).

For an edge shared by (k1, f1) and (k2, f2), with e1 -> e2 the face as traversed
counter-clockwise by element k1 and q1, q2 the two apexes:

1. Enclosed parallelogram (Sec. 4.2).  It shares the diagonal e1e2.  Reflecting T2 about
   the edge midpoint c maps it onto a triangle over the same base on T1's side; any
   parallelogram with diagonal e1e2 inside T1 u T2 has one apex p1 in T1 and p2 = 2c - p1
   in T2, i.e. p1 in T1 n (2c - T2).  The reading taken is the maximum-area one: p1 is the
   point of that intersection (clipped with Sutherland-Hodgman) farthest from e1e2.
2. Projection (Eqs. NodalToModalProjection, changeOfHypotenuseProjection,
   totalProjection): u_hat'_k = V^{-1} V_pk V_rfk^{-1} u_k, where V_rfk is the rotation
   Vandermonde of face f_k and V_pk evaluates the rotated-frame modal expansion at the
   nodes of the sub-triangle Omega'_k = (p_k, face first vertex, face second vertex).
3. Reconstruction (Sec. 4.5): least squares of the 2 Np weak equalities over the tensor
   Legendre basis on the logical square, side 1 on I (parallelogram coordinates (R,S) =
   side 1's rotated frame) and side 2 on I^{-1} ((R,S) = -(r,s) of side 2's rotated frame,
   the point reflection that maps e1, e2, p2 correctly).
4. Edge gradient: grad u~ = [R_x S_x; R_y S_y] [d_R u~; d_S u~] with the constant metric of
   Omega'_1 (x_R = (e1-p1)/2, x_S = (e2-p1)/2), evaluated at the diagonal nodes
   (R,S) = (-t, t), t the LGL points, in side 1's face order; g = n1 . grad u~.
5. Algorithm 2 for element-wise D: D~ = RDG(D1, D2) with the same operators, evaluated at
   the diagonal nodes.
"""
from __future__ import annotations

import numpy as np

from .mesh import FACE_APEX, FACE_VERTS, Mesh
from .refops import psi


def _clip(poly, a, b):
    """Keep the part of polygon `poly` on the left of the directed line a -> b."""
    out = []
    n = len(poly)
    side = lambda p: (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])
    for i in range(n):
        P, Q = poly[i], poly[(i + 1) % n]
        sp, sq = side(P), side(Q)
        if sp >= 0:
            out.append(P)
        if (sp >= 0) != (sq >= 0):
            t = sp / (sp - sq)
            out.append(P + t * (Q - P))
    return out


def enclosed_parallelogram(e1, e2, q1, q2):
    """Apexes (p1, p2) of the maximum-area parallelogram with diagonal e1e2 enclosed in the
    quadrilateral (e1, q2, e2, q1) formed by triangles T1 = (e1, e2, q1), T2 = (e2, e1, q2)."""
    c = (e1 + e2) / 2
    T1 = [np.array(e1, float), np.array(e2, float), np.array(q1, float)]
    T2r = [2 * c - np.array(e2, float), 2 * c - np.array(e1, float), 2 * c - np.array(q2, float)]   # = (e1, e2, 2c-q2)
    poly = T1
    for i in range(3):
        poly = _clip(poly, T2r[i], T2r[(i + 1) % 3])
    d = e2 - e1
    height = lambda p: (d[0] * (p[1] - e1[1]) - d[1] * (p[0] - e1[0]))
    p1 = max(poly, key=height)
    return p1, 2 * c - p1


def rotated_frame_coords(va, vb, vc, p):
    """(r, s) of physical point p in the frame that puts va at (1,-1), vb at (-1,1) and
    the apex vc at (-1,-1):  p = -(r+s)/2 vc + (r+1)/2 va + (s+1)/2 vb."""
    Amat = np.column_stack([(va - vc) / 2, (vb - vc) / 2])
    rhs = p - (va + vb) / 2
    return np.linalg.solve(Amat, rhs)


class EdgeOps:
    """Per-edge setup quantities for a mesh (parallelogram, projections, metric)."""

    def __init__(self, mesh: Mesh):
        self.mesh = mesh
        ops = mesh.ops
        E = mesh.E
        Np = ops.Np
        self.p1 = np.zeros((E, 2))
        self.p2 = np.zeros((E, 2))
        self.ab1 = np.zeros((E, 2))
        self.ab2 = np.zeros((E, 2))
        self.P1 = np.zeros((E, Np, Np))
        self.P2 = np.zeros((E, Np, Np))
        self.n1 = np.zeros((E, 2))
        self.Rx = np.zeros((E, 4))      # R_x, R_y, S_x, S_y
        self.e1 = np.zeros((E, 2))
        self.e2 = np.zeros((E, 2))
        for e, (k1, f1, k2, f2, shx, shy) in enumerate(mesh.edges):
            a1, b1 = FACE_VERTS[f1]
            e1 = mesh.V[k1, a1]
            e2 = mesh.V[k1, b1]
            q1 = mesh.V[k1, FACE_APEX[f1]]
            if k2 >= 0:
                q2 = mesh.V[k2, FACE_APEX[f2]] + np.array([shx, shy])
            else:
                q2 = e1 + e2 - q1           # ghost: reflected apex
            p1, p2 = enclosed_parallelogram(e1, e2, q1, q2)
            self.p1[e], self.p2[e], self.e1[e], self.e2[e] = p1, p2, e1, e2
            # side 1 frame: face first vertex e1, second e2, apex q1
            self.ab1[e] = rotated_frame_coords(e1, e2, q1, p1)
            # side 2 frame: element k2 traverses the face e2 -> e1
            self.ab2[e] = rotated_frame_coords(e2, e1, q2, p2)
            self.P1[e] = self.projection(self.ab1[e], f1)
            self.P2[e] = self.projection(self.ab2[e], f2 if k2 >= 0 else 1)
            # side 1 outward normal and parallelogram metric (constant)
            d = e2 - e1
            self.n1[e] = np.array([d[1], -d[0]]) / np.hypot(*d)
            xR, yR = (e1 - p1) / 2
            xS, yS = (e2 - p1) / 2
            Jp = xR * yS - xS * yR
            self.Rx[e] = [yS / Jp, -xS / Jp, -yR / Jp, xR / Jp]

    def projection(self, ab, f):
        """V^{-1} V_p V_rf^{-1} (Eq. totalProjection) for apex coordinates ab in the frame of
        face f.  V_p[i, j] = psi_j(A(r_i, s_i)), A mapping I onto Omega' in that frame."""
        ops = self.mesh.ops
        r, s = ops.r, ops.s
        al, be = ab
        Ar = -(r + s) / 2 * al + (r + 1) / 2 * 1.0 + (s + 1) / 2 * (-1.0)
        As = -(r + s) / 2 * be + (r + 1) / 2 * (-1.0) + (s + 1) / 2 * 1.0
        Vp = psi(ops.N, Ar, As)
        return ops.Vinv @ Vp @ ops.Vr_inv[f]

    # -- reconstruction and edge gradient ----------------------------------------------
    def reconstruct(self, u1, u2):
        """Reconstructed tensor-Legendre coefficients c [E, Mp] from side nodal values
        u1, u2 [E, Np] (Algorithm aRDG then least squares)."""
        uh1 = np.einsum("eij,ej->ei", self.P1, u1)
        uh2 = np.einsum("eij,ej->ei", self.P2, u2)
        rhs = np.concatenate([uh1, uh2], axis=1)
        return rhs @ self.mesh.ops.Apinv.T

    def edge_gradient(self, c):
        """(d/dx u~, d/dy u~) [E, Nfp] at the diagonal nodes (side 1 face order)."""
        ops = self.mesh.ops
        dR = c @ ops.DR.T
        dS = c @ ops.DS.T
        Rx, Ry, Sx, Sy = self.Rx.T
        ux = Rx[:, None] * dR + Sx[:, None] * dS
        uy = Ry[:, None] * dR + Sy[:, None] * dS
        return ux, uy

    def edge_normal_gradient(self, c):
        """g[e, i] = n1 . grad u~ at the diagonal nodes (side 1 face order)."""
        ux, uy = self.edge_gradient(c)
        return self.n1[:, 0:1] * ux + self.n1[:, 1:2] * uy

    def reconstructed_values(self, c):
        """u~ at the diagonal nodes."""
        ops = self.mesh.ops
        return c @ ops.phi(ops.diag_R, ops.diag_S).T

    def flux_algorithm1(self, c, D1, D2):
        """Algorithm 1 (Sec. 3, Eq. NDG_diffusion_once_matrixForm_reference_general) for
        element-constant D: n1 . RDG(D_p^1 grad u~^1, D_p^2 grad u~^2) at the diagonal nodes.

        The steps in the paper's order, for reconstruction coefficients c [E, Mp] of u~:
        Separation - u~ L2-projected onto P_N on each sub-triangle Omega'_k, in side k's frame
        (side 1: (r,s) = (R,S); side 2: (r,s) = (-R,-S)): modal coefficients A_k c.
        D_p^k = V_pk D^k - the projection of an element-constant D is that constant.
        Grad - nodal gradient of u~^k on Omega'_k in physical coordinates, d/dR = +-d/dr.
        Product - D_p^k grad u~^k at the sub-triangle nodes.
        RDG - least-squares reconstruction of each component from the two sub-triangles'
        modal data, evaluated at the diagonal nodes; then n1 . (.).

        D1, D2 are [E] (isotropic), [E, 2] (the diagonal tensor (Dx, Dy) of Eq.
        NDG_diffusion_once_matrixForm_reference_general: component x of the product uses Dx),
        or [E, Np] (nodal values of a spatially varying D on each side's element, in the
        element's own node order): then D_p^k = V_pk D^k is the element's D evaluated at the
        nodes of the sub-triangle, V (P_k D^k) with the projection P_k of Eq. totalProjection."""
        ops = self.mesh.ops
        Rx, Ry, Sx, Sy = self.Rx.T
        Phi = ops.phi(ops.diag_R, ops.diag_S)
        out = np.zeros((c.shape[0], ops.Nfp))
        nodal = np.asarray(D1).ndim == 2 and np.asarray(D1).shape[1] == ops.Np
        if nodal:   # D_p^k at the sub-triangle nodes
            D1 = np.einsum("ij,ejk,ek->ei", ops.V, self.P1, np.asarray(D1))
            D2 = np.einsum("ij,ejk,ek->ei", ops.V, self.P2, np.asarray(D2))
        for comp in range(2):
            dRphys = Rx if comp == 0 else Ry     # d/dx = R_x d/dR + S_x d/dS (y likewise)
            dSphys = Sx if comp == 0 else Sy
            modal = []
            for side, (Ak, sgn, Dk) in enumerate(((ops.A1, 1.0, D1), (ops.A2, -1.0, D2))):
                uk = c @ Ak.T                       # Separation: modal on Omega'_k [E, Np]
                nod = uk @ ops.V.T                  # nodal values at the sub-triangle nodes
                dr = nod @ ops.Dr.T
                ds = nod @ ops.Ds.T
                g = sgn * (dRphys[:, None] * dr + dSphys[:, None] * ds)
                Dc = np.asarray(Dk)
                if nodal:
                    w = Dc * g                      # Product with D_p^k at the nodes
                else:
                    Dc = Dc[:, comp] if Dc.ndim == 2 else Dc
                    w = Dc[:, None] * g             # Product with D_p^k (component comp)
                modal.append(w @ ops.Vinv.T)        # modal data of the component on Omega'_k
            cc = np.concatenate(modal, axis=1) @ ops.Apinv.T   # RDG of the component
            out += self.n1[:, comp:comp + 1] * (cc @ Phi.T)
        return out

    def reconstruct_D(self, D1, D2):
        """Algorithm 2: D~ = RDG(D1, D2) for element-constant D, values at diagonal nodes."""
        Np = self.mesh.ops.Np
        u1 = np.outer(D1, np.ones(Np))
        u2 = np.outer(D2, np.ones(Np))
        return self.reconstructed_values(self.reconstruct(u1, u2))
