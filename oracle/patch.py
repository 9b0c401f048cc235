"""The oracle on sampled elements of a mesh too large for it (test infrastructure only).

The semi-discrete right-hand side of element k (Eq. NDG_diffusion_once_matrixForm_Fullyreference)
reads the state of k and of its three face neighbours only: the volume term reads u_k, and
the flux of each of k's edges is built from the two elements that share it (the
reconstruction on the enclosed parallelogram, Sec. 4 and Algorithm aRDG).  An SSP-RK3 step
has three such stages, so the step's result on k reads the elements up to three faces away.

So the oracle's result on a set S of sampled elements of a large periodic mesh is the
oracle's result on a small patch: the elements within `rings` faces of S, each placed at the
periodic image that makes it touch the element it was reached from, taken as a mesh of its
own (the patch's outer faces become boundary edges whose ghost data is zero).  Wrong values
enter only through those outer faces, one ring per stage, so with rings >= stages they never
reach S.  An element reached through two different periodic images is placed twice (once
per image); distinct (element, image) pairs never overlap because the mesh tiles the torus.

Only the element neighbourhood search and the placement live here; every number comes from
``oracle.mesh.Mesh`` and ``oracle.rhs.Problem`` on the patch.
"""
from __future__ import annotations

import numpy as np

from .mesh import DIRICHLET, FACE_VERTS, PERIODIC, Mesh
from .rhs import Problem


def face_neighbours(xy, tri, bc=PERIODIC, period=(1.0, 1.0)):
    """Face neighbour of every (element, face) and the translation that brings the neighbour
    onto the shared face: nbr [K, 3] (-1 on a Dirichlet boundary), shift [K, 3, 2].  Faces are
    matched by their midpoints, modulo the period on a periodic mesh (as ``Mesh`` does)."""
    V = np.asarray(xy, float)[np.asarray(tri, np.int64)]
    K = V.shape[0]
    per = np.asarray(period, float)
    mids = np.stack([(V[:, a] + V[:, b]) / 2 for a, b in FACE_VERTS], axis=1)      # [K, 3, 2]
    q = mids.reshape(-1, 2)
    if bc == PERIODIC:
        q = np.mod(q, per)
        q = np.where(np.abs(q - per) < 1e-9, 0.0, q)
        key = np.round(q * 1e9).astype(np.int64)
    else:
        key = np.round(q * 1e12).astype(np.int64)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    inv = inv.ravel()
    if np.any(cnt > 2):
        raise ValueError("non-manifold edge")
    order = np.argsort(inv, kind="stable")
    si = inv[order]
    nbr = -np.ones(3 * K, np.int64)
    pair = np.flatnonzero(si[1:] == si[:-1])
    a, b = order[pair], order[pair + 1]
    nbr[a], nbr[b] = b, a
    if bc == PERIODIC and np.any(nbr < 0):
        raise ValueError("unmatched face on a periodic mesh")
    shift = np.zeros((3 * K, 2))
    has = nbr >= 0
    shift[has] = q_raw = mids.reshape(-1, 2)[has] - mids.reshape(-1, 2)[nbr[has]]
    if bc == PERIODIC:                         # a whole number of periods, exactly
        shift[has] = np.round(q_raw / per) * per
    nk = np.where(has, nbr // 3, -1)
    return nk.reshape(K, 3), shift.reshape(K, 3, 2)


def build_patch(xy, tri, sample, rings, bc=PERIODIC, period=(1.0, 1.0), nbr=None):
    """Elements within `rings` faces of `sample`, as (orig [P], shift [P, 2]); the sampled
    elements come first, in the given order, at zero shift."""
    if nbr is None:
        nbr = face_neighbours(xy, tri, bc, period)
    nk, sh = nbr
    per = np.asarray(period, float)
    seen = {}
    orig, shift = [], []

    def add(k, d):
        key = (int(k), int(round(d[0] / per[0])), int(round(d[1] / per[1])))
        if key in seen:
            return False
        seen[key] = len(orig)
        orig.append(int(k))
        shift.append(np.array([key[1] * per[0], key[2] * per[1]]))
        return True

    front = []
    for k in sample:
        if add(k, (0.0, 0.0)):
            front.append(len(orig) - 1)
    for _ in range(rings):
        nxt = []
        for i in front:
            k, d = orig[i], shift[i]
            for f in range(3):
                n = nk[k, f]
                if n >= 0 and add(n, d + sh[k, f]):
                    nxt.append(len(orig) - 1)
        front = nxt
    return np.array(orig, np.int64), np.array(shift)


class PatchProblem:
    """The oracle Problem on the patch around `sample`: rhs and rk3_step on full-mesh nodal
    arrays, returning the rows of the sampled elements only."""

    def __init__(self, xy, tri, N, D_elem, sample, v=(0.0, 0.0), rings=1, interface="alg2",
                 period=(1.0, 1.0), nbr=None):
        xy = np.asarray(xy, float)
        tri = np.asarray(tri, np.int64)
        self.sample = np.asarray(sample, np.int64)
        if np.unique(self.sample).size != self.sample.size:
            raise ValueError("sampled elements must be distinct")
        self.orig, shift = build_patch(xy, tri, self.sample, rings, PERIODIC, period, nbr)
        P = self.orig.size
        Vp = xy[tri[self.orig]] + shift[:, None, :]                      # [P, 3, 2]
        pxy = Vp.reshape(-1, 2)
        ptri = np.arange(3 * P).reshape(P, 3)
        self.mesh = Mesh(pxy, ptri, N, bc=DIRICHLET)
        D = np.asarray(D_elem, float)
        Dp = D[self.orig] if D.ndim else np.full(P, float(D))
        self.problem = Problem(self.mesh, Dp, v=v, ghost_fn=lambda x, y, t: 0.0 * x, interface=interface)
        self.ns = self.sample.size
        self.patch_elements = P

    def rhs(self, u_full, t=0.0):
        return self.problem.rhs(np.asarray(u_full, float)[self.orig], t)[: self.ns]

    def rk3_step(self, u_full, t, dt):
        return self.problem.rk3_step(np.asarray(u_full, float)[self.orig], t, dt)[: self.ns]
