"""Mesh connectivity and affine element geometry for the oracle (test infrastructure only).

Affine triangle map x = -(r+s)/2 v1 + (r+1)/2 v2 + (s+1)/2 v3 (Eq. mapping_tri) with
constant metric terms rx = ys/J, ry = -xs/J, sx = -yr/J, sy = xr/J, J = xr ys - xs yr
(Eqs. mapping_tri_diff, triangle_jacobian).  Edge Jacobian J_f = |edge|/2 (Eq.
lift_physicalDomain_ardg: the ratio of edge length to the reference edge length 2).

Edges are found by matching face midpoints; with periodic boundaries the midpoints are
taken modulo the period and side 2's coordinates are translated so its face coincides with
side 1's.  With Dirichlet boundaries every unmatched face becomes a boundary edge whose
side 2 is the ghost triangle obtained by point reflection of the element about the edge
midpoint (a reading: the paper does not discuss boundaries).
"""
from __future__ import annotations

import numpy as np

from .refops import RefOps

PERIODIC = 0
DIRICHLET = 1

FACE_VERTS = [(0, 1), (1, 2), (2, 0)]   # faces 1, 2, 3 as (first, second) vertex slots
FACE_APEX = [2, 0, 1]


class Mesh:
    def __init__(self, xy, tri, N: int, bc: int = PERIODIC, period=(1.0, 1.0)):
        self.xy = np.asarray(xy, float)
        self.tri = np.asarray(tri, np.int64)
        self.K = self.tri.shape[0]
        self.bc = bc
        self.period = np.asarray(period, float)
        self.ops = RefOps(N)
        self.V = self.xy[self.tri]            # [K, 3, 2] element vertex coordinates
        self._geometry()
        self._connect()

    # --------------------------------------------------------------------------------
    def _geometry(self):
        v1, v2, v3 = self.V[:, 0], self.V[:, 1], self.V[:, 2]
        xr, yr = ((v2 - v1) / 2).T
        xs, ys = ((v3 - v1) / 2).T
        self.J = xr * ys - xs * yr
        if np.any(self.J <= 0):
            raise ValueError("mesh has a triangle that is not counter-clockwise or is degenerate")
        self.rx, self.ry = ys / self.J, -xs / self.J
        self.sx, self.sy = -yr / self.J, xr / self.J
        # physical node coordinates
        r, s = self.ops.r, self.ops.s
        self.x = np.outer(-(r + s) / 2, v1[:, 0]).T + np.outer((r + 1) / 2, v2[:, 0]).T + np.outer((s + 1) / 2, v3[:, 0]).T
        self.y = np.outer(-(r + s) / 2, v1[:, 1]).T + np.outer((r + 1) / 2, v2[:, 1]).T + np.outer((s + 1) / 2, v3[:, 1]).T
        # outward unit normals, edge Jacobians and Fscale per face
        self.nx = np.zeros((self.K, 3))
        self.ny = np.zeros((self.K, 3))
        self.sJ = np.zeros((self.K, 3))
        for f, (a, b) in enumerate(FACE_VERTS):
            d = self.V[:, b] - self.V[:, a]
            ln = np.hypot(d[:, 0], d[:, 1])
            self.nx[:, f] = d[:, 1] / ln
            self.ny[:, f] = -d[:, 0] / ln
            self.sJ[:, f] = ln / 2
        self.Fscale = self.sJ / self.J[:, None]

    def _canon(self, p):
        """Canonical representative of a point (periodic identification)."""
        if self.bc == PERIODIC:
            q = np.mod(p, self.period)
            q = np.where(np.abs(q - self.period) < 1e-9, 0.0, q)
            return (round(q[0] * 1e9), round(q[1] * 1e9))
        return (round(p[0] * 1e12), round(p[1] * 1e12))

    def _connect(self):
        table = {}
        for k in range(self.K):
            for f, (a, b) in enumerate(FACE_VERTS):
                # an edge is identified by its midpoint (modulo the period): two faces
                # meet there exactly when they are the same edge of a conforming mesh
                key = self._canon((self.V[k, a] + self.V[k, b]) / 2)
                table.setdefault(key, []).append((k, f))
        edges = []        # (k1, f1, k2, f2, shift_x, shift_y); k2 = -1 for boundary
        for key, lst in table.items():
            if len(lst) == 2:
                (k1, f1), (k2, f2) = sorted(lst)
                a1, b1 = FACE_VERTS[f1]
                a2, b2 = FACE_VERTS[f2]
                mid1 = (self.V[k1, a1] + self.V[k1, b1]) / 2
                mid2 = (self.V[k2, a2] + self.V[k2, b2]) / 2
                sh = mid1 - mid2
                edges.append((k1, f1, k2, f2, sh[0], sh[1]))
            elif len(lst) == 1:
                if self.bc == PERIODIC:
                    raise ValueError("unmatched face on a periodic mesh")
                k1, f1 = lst[0]
                edges.append((k1, f1, -1, -1, 0.0, 0.0))
            else:
                raise ValueError("non-manifold edge")
        edges.sort(key=lambda e: (e[2] < 0, e[0], e[1]))
        self.edges = edges
        self.E = len(edges)
        self.n_interior = sum(1 for e in edges if e[2] >= 0)
        # element face -> (edge, side)
        self.elem_edge = np.zeros((self.K, 3, 2), np.int64)
        for e, (k1, f1, k2, f2, _, _) in enumerate(edges):
            self.elem_edge[k1, f1] = (e, 1)
            if k2 >= 0:
                self.elem_edge[k2, f2] = (e, 2)

    # --------------------------------------------------------------------------------
    def ghost_vertices(self, e):
        """Ghost triangle of boundary edge e in standard vertex slots: v1 = reflected apex,
        v2 = the face's second vertex, v3 = its first (face 2 = hypotenuse is the shared
        edge traversed in the opposite direction, so the ghost is counter-clockwise)."""
        k1, f1 = self.edges[e][0], self.edges[e][1]
        a, b = FACE_VERTS[f1]
        e1, e2, q1 = self.V[k1, a], self.V[k1, b], self.V[k1, FACE_APEX[f1]]
        return np.stack([e1 + e2 - q1, e2, e1])

    def ghost_nodes(self, e):
        g = self.ghost_vertices(e)
        r, s = self.ops.r, self.ops.s
        pts = np.outer(-(r + s) / 2, g[0]) + np.outer((r + 1) / 2, g[1]) + np.outer((s + 1) / 2, g[2])
        return pts[:, 0], pts[:, 1]

    def boundary_edges(self):
        return [e for e in range(self.E) if self.edges[e][2] < 0]

    def element_area(self):
        return 2.0 * self.J
