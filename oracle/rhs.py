"""Semi-discrete right-hand side, SSP-RK3 and error norms, oracle version (test
infrastructure only).

The weak form of u_t + div(v u) - div(D grad u) = s (Eq. convection_diffusion) on element
k, with F = v u - D grad u, reads (Eq. NDG_diffusion_once_matrixForm_Fullyreference for
v = 0, constant D):

    du/dt = M^{-1} S^T . F  -  sum_f (J_f / J) LIFT_f (F* . n)_f  +  s

with the reference matrices of Sec. 3, the volume flux F interpolated at the nodes, and
the interface flux F*.n = (v.n) u_upwind - D~ n.grad u~ at the face nodes: grad u~ from the
parallelogram reconstruction, D~ from Algorithm 2 (element-wise D), u_upwind the trace on
the upwind side (a reading: the paper does not fix the convective flux for this equation).
For D constant and v = 0 this is exactly the paper's equation.

The time integrator is the three-stage SSP-RK3 scheme (the paper itself uses a five-stage
fourth-order low-storage scheme); error norms follow Eqs. L2_norm_cellUnit and
Linf_norm_cellUnit (the "L_inf" norm is a maximum of cell means).
"""
from __future__ import annotations

import math

import numpy as np

from synth import tau as _tau
from .ardg import EdgeOps
from .mesh import FACE_VERTS, Mesh
from .refops import psi, triangle_quadrature


# Published coefficients of the five-stage fourth-order 2N-storage Runge-Kutta scheme
# (Carpenter and Kennedy 1994, solution 3), the integrator of the paper's Sec. 5.
LSRK_A = (0.0,
          -567301805773.0 / 1357537059087.0,
          -2404267990393.0 / 2016746695238.0,
          -3550918686646.0 / 2091501179385.0,
          -1275806237668.0 / 842570457699.0)
LSRK_B = (1432997174477.0 / 9575080441755.0,
          5161836677717.0 / 13612068292357.0,
          1720146321549.0 / 2090206949498.0,
          3134564353537.0 / 4481467310338.0,
          2277821191437.0 / 14882151754819.0)
LSRK_C = (0.0,
          1432997174477.0 / 9575080441755.0,
          2526269341429.0 / 6820363962896.0,
          2006345519317.0 / 3224310063776.0,
          2802321613138.0 / 2924317926251.0)


class Problem:
    """A mesh plus coefficients: D per element, constant velocity v, optional separable
    source and Dirichlet ghost data (lists of (nodal profile, kind, omega)).

    D_elem: [K] for isotropic diffusion, [K, 2] for the diagonal tensor D = (Dx, Dy) of Eq.
    NDG_diffusion_once_matrixForm_reference_general (the volume flux is (Dx u_x, Dy u_y); the
    interface rules below act on each component), or [K, Np] for a spatially varying D given
    at the nodes (the volume flux is the nodal product D grad u; Algorithm 2 reconstructs D~
    from both elements' nodal D, the harmonic rule takes the harmonic mean of the two traces,
    Algorithm 1 evaluates each element's D at its sub-triangle's nodes).  A Dirichlet ghost's
    nodal D is its element's D at the reflected points.

    interface: how the edge diffusion coefficient D~ is formed for element-wise D.
      "alg1"      the paper's Algorithm 1: the edge flux is n . RDG(D_p^1 grad u~^1,
                  D_p^2 grad u~^2) with Separation read as the L2 projection of u~ onto
                  each sub-triangle (EdgeOps.flux_algorithm1);
      "alg2"      the paper's Algorithm 2, D~ = RDG(D1, D2) on the diagonal;
      "harmonic"  2 D1 D2 / (D1 + D2), not in the paper: a stabilised variant for
                  high-contrast jumps (with "alg2" such jumps give operator eigenvalues with
                  positive real part).  Both equal D when D1 = D2.
    """

    def __init__(self, mesh: Mesh, D_elem, v=(0.0, 0.0), source=None, ghost_fn=None, interface="alg2"):
        self.mesh = mesh
        self.eops = EdgeOps(mesh)
        self.D = np.asarray(D_elem, float)
        self.v = np.asarray(v, float)
        self.source = source or []       # list of (S [K,Np], kind, omega)
        self.ghost_fn = ghost_fn         # callable(x, y, t) for Dirichlet ghost values
        m = mesh
        self.k1 = np.array([e[0] for e in m.edges])
        self.f1 = np.array([e[1] for e in m.edges])
        self.k2 = np.array([e[2] for e in m.edges])
        self.f2 = np.array([e[3] for e in m.edges])
        self.interior = self.k2 >= 0
        ops = m.ops
        self.nodal = self.D.ndim == 2 and self.D.shape[1] == ops.Np
        self.aniso = self.D.ndim == 2 and not self.nodal
        if self.aniso and self.D.shape[1] != 2:
            raise ValueError("D_elem must be [K], [K, 2] or [K, Np]")
        self.bnd = np.flatnonzero(~self.interior)
        self.ghost_xy = [m.ghost_nodes(e) for e in self.bnd]
        inner = self.interior[:, None] if self.D.ndim == 2 else self.interior
        D2 = np.where(inner, self.D[np.maximum(self.k2, 0)], self.D[self.k1])
        if self.nodal and self.bnd.size:
            D2[self.bnd] = self._ghost_D()
        self.interface = interface
        self.D1e, self.D2e = self.D[self.k1], D2
        comps = [(self.D1e[:, c], D2[:, c]) for c in range(2)] if self.aniso else [(self.D1e, D2)]
        if interface == "alg1":
            self.Dt = None
        elif interface == "alg2" and self.nodal:
            self.Dt = self.eops.reconstructed_values(self.eops.reconstruct(self.D1e, D2))
        elif interface == "alg2":
            self.Dt = [self.eops.reconstruct_D(a, b) for a, b in comps]
        elif interface == "harmonic" and self.nodal:
            t1 = np.take_along_axis(self.D1e, np.stack([ops.Fmask[f] for f in self.f1]), axis=1)
            f2i = np.where(self.interior, self.f2, 1)
            t2 = np.take_along_axis(D2, np.stack([ops.Fmask[f][::-1] for f in f2i]), axis=1)
            self.Dt = 2 * t1 * t2 / (t1 + t2)
        elif interface == "harmonic":
            self.Dt = [np.repeat((2 * a * b / (a + b))[:, None], mesh.ops.Nfp, axis=1) for a, b in comps]
        else:
            raise ValueError(interface)
        if not self.aniso and not self.nodal and self.Dt is not None:
            self.Dt = self.Dt[0]

    def _ghost_D(self):
        """Nodal D of every ghost: its element's D at the point reflections of the ghost's nodes
        (the ghost is the element reflected about the edge midpoint)."""
        m = self.mesh
        ops = m.ops
        out = np.zeros((self.bnd.size, ops.Np))
        for i, e in enumerate(self.bnd):
            k1, f1 = self.k1[e], self.f1[e]
            a, b = FACE_VERTS[f1]
            c2 = m.V[k1, a] + m.V[k1, b]
            gx, gy = self.ghost_xy[i]
            px, py = c2[0] - gx, c2[1] - gy
            v1, v2, v3 = m.V[k1]
            Amat = np.column_stack([(v2 - v1) / 2, (v3 - v1) / 2])
            rs = np.linalg.solve(Amat, np.stack([px - (v2[0] + v3[0]) / 2, py - (v2[1] + v3[1]) / 2]))
            out[i] = psi(ops.N, rs[0], rs[1]) @ (ops.Vinv @ self.D[k1])
        return out

    def ghost_values(self, t):
        Np = self.mesh.ops.Np
        out = np.zeros((self.bnd.size, Np))
        for i, (gx, gy) in enumerate(self.ghost_xy):
            out[i] = self.ghost_fn(gx, gy, t)
        return out

    def edge_flux(self, u, t=0.0):
        """F*.n1 at the face nodes of every edge, side 1's face order: [E, Nfp]."""
        m = self.mesh
        ops = m.ops
        u1 = u[self.k1]
        u2 = np.zeros_like(u1)
        u2[self.interior] = u[self.k2[self.interior]]
        if self.bnd.size:
            u2[self.bnd] = self.ghost_values(t)
        c = self.eops.reconstruct(u1, u2)
        if self.interface == "alg1":
            Dg = self.eops.flux_algorithm1(c, self.D1e, self.D2e)
        elif self.aniso:
            ux, uy = self.eops.edge_gradient(c)       # n1 . (D~x u~_x, D~y u~_y)
            Dg = self.eops.n1[:, 0:1] * self.Dt[0] * ux + self.eops.n1[:, 1:2] * self.Dt[1] * uy
        else:
            Dg = self.Dt * self.eops.edge_normal_gradient(c)
        # upwind convective trace
        vn = self.eops.n1 @ self.v
        tr1 = np.take_along_axis(u1, np.stack([ops.Fmask[f] for f in self.f1]), axis=1)
        f2i = np.where(self.interior, self.f2, 1)
        tr2 = np.take_along_axis(u2, np.stack([ops.Fmask[f][::-1] for f in f2i]), axis=1)
        up = np.where((vn >= 0)[:, None], tr1, tr2)
        return vn[:, None] * up - Dg

    def rhs(self, u, t=0.0):
        m = self.mesh
        ops = m.ops
        if self.nodal:
            Dx = Dy = self.D
        else:
            Dx = (self.D[:, 0] if self.aniso else self.D)[:, None]
            Dy = (self.D[:, 1] if self.aniso else self.D)[:, None]
        ur = u @ ops.Dr.T
        us = u @ ops.Ds.T
        ux = m.rx[:, None] * ur + m.sx[:, None] * us
        uy = m.ry[:, None] * ur + m.sy[:, None] * us
        Fx = self.v[0] * u - Dx * ux
        Fy = self.v[1] * u - Dy * uy
        # volume term M^{-1} S^T . F  (S = J r_x S_ref, the J cancels with M^k = J M)
        Fr = m.rx[:, None] * Fx + m.ry[:, None] * Fy
        Fs = m.sx[:, None] * Fx + m.sy[:, None] * Fy
        out = (Fr @ ops.Sr + Fs @ ops.Ss) @ ops.Minv.T
        # surface term
        fl = self.edge_flux(u, t)
        # side 1 takes F*.n1 in its face order; side 2 (n2 = -n1, face traversed the other
        # way) takes -F*.n1 reversed
        q1 = fl
        c1 = m.Fscale[self.k1, self.f1][:, None] * np.einsum("eiq,eq->ei", ops.LIFT[self.f1], q1)
        np.add.at(out, self.k1, -c1)
        ii = np.flatnonzero(self.interior)
        q2 = -fl[ii][:, ::-1]
        k2, f2 = self.k2[ii], self.f2[ii]
        c2 = m.Fscale[k2, f2][:, None] * np.einsum("eiq,eq->ei", ops.LIFT[f2], q2)
        np.add.at(out, k2, -c2)
        for S, kind, om in self.source:
            out += _tau(kind, om, t) * S
        return out

    def rk3_step(self, u, t, dt):
        """One SSP-RK3 step: stages at t, t+dt, t+dt/2."""
        u1 = u + dt * self.rhs(u, t)
        u2 = 0.75 * u + 0.25 * (u1 + dt * self.rhs(u1, t + dt))
        return u / 3.0 + 2.0 / 3.0 * (u2 + dt * self.rhs(u2, t + 0.5 * dt))

    def lsrk_step(self, u, t, dt):
        """One step of the five-stage fourth-order low-storage Runge-Kutta scheme the paper
        uses (Sec. 5, Carpenter and Kennedy 1994), in its two-register form: for stage i,
        du = a_i du + dt L(u, t + c_i dt), u = u + b_i du."""
        du = np.zeros_like(u)
        for a, b, c in zip(LSRK_A, LSRK_B, LSRK_C):
            du = a * du + dt * self.rhs(u, t + c * dt)
            u = u + b * du
        return u

    def solve(self, u, t0, dt, nsteps, scheme="ssp3"):
        step = self.rk3_step if scheme == "ssp3" else self.lsrk_step
        for n in range(nsteps):
            u = step(u, t0 + n * dt, dt)
        return u

    def dense_operator(self):
        """L[:, j] = rhs(e_j) with no forcing (column by column)."""
        K, Np = self.mesh.K, self.mesh.ops.Np
        n = K * Np
        Lop = np.zeros((n, n))
        save_src = self.source
        self.source = []
        try:
            for j in range(n):
                ej = np.zeros(n)
                ej[j] = 1.0
                Lop[:, j] = self.rhs(ej.reshape(K, Np), 0.0).ravel()
        finally:
            self.source = save_src
        return Lop


def nodal(mesh: Mesh, fn, *args):
    return fn(mesh.x, mesh.y, *args)


def error_norms(mesh: Mesh, u, exact_fn, t):
    """(L2, L_inf-of-cell-means) of u - u_e with a degree 2N+4 rule on each element."""
    ops = mesh.ops
    rq, sq, wq = triangle_quadrature(2 * ops.N + 4)
    interp = psi(ops.N, rq, sq) @ ops.Vinv        # nodal -> quadrature points
    v1, v2, v3 = mesh.V[:, 0], mesh.V[:, 1], mesh.V[:, 2]
    xq = np.outer(-(rq + sq) / 2, v1[:, 0]).T + np.outer((rq + 1) / 2, v2[:, 0]).T + np.outer((sq + 1) / 2, v3[:, 0]).T
    yq = np.outer(-(rq + sq) / 2, v1[:, 1]).T + np.outer((rq + 1) / 2, v2[:, 1]).T + np.outer((sq + 1) / 2, v3[:, 1]).T
    err = u @ interp.T - exact_fn(xq, yq, t)
    area = 2.0 * mesh.J
    l2 = math.sqrt(np.sum(mesh.J[:, None] * wq[None, :] * err ** 2) / np.sum(area))
    cellmean = np.sum(mesh.J[:, None] * wq[None, :] * np.abs(err), axis=1) / area
    return l2, float(np.max(cellmean))


def power_spectral_radius(prob: Problem, iters: int = 50, seed: int = 0):
    """Estimate rho(L) by normalised power iteration on the RHS operator (no forcing)."""
    K, Np = prob.mesh.K, prob.mesh.ops.Np
    x = np.random.default_rng(seed).standard_normal((K, Np))
    save_src, save_g = prob.source, prob.ghost_fn
    prob.source = []
    if prob.ghost_fn is not None:
        prob.ghost_fn = lambda X, Y, t: 0.0 * X
    rho = 0.0
    try:
        for _ in range(iters):
            x /= np.linalg.norm(x)
            y = prob.rhs(x, 0.0)
            rho = np.linalg.norm(y)
            x = y
    finally:
        prob.source, prob.ghost_fn = save_src, save_g
    return rho


SSP_RK3_NEG_REAL_EXTENT = 2.5127


def stable_dt(prob: Problem, factor=0.5, iters=50, seed=0):
    return factor * SSP_RK3_NEG_REAL_EXTENT / power_spectral_radius(prob, iters, seed)
