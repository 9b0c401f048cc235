"""Seeded synthetic inputs shared by the CUDA library's tests/bench and the oracle.

This module holds input definitions only: mesh vertex/triangle arrays, per-element
coefficients, closed-form initial/exact/source functions of (x, y, t) and seeded random
nodal fields.  It contains none of the reconstructed-DG arithmetic (no nodes, no
operators, no reconstruction): each side evaluates the functions given here at its own
node coordinates.

Mesh recipe (the paper's grids a/b/c are not available, so these stand in for them):
the unit square is cut into m x m cells, each cell split by its "/" diagonal into two
counter-clockwise triangles; interior vertices are moved by
``default_rng(seed).uniform(-jitter*h, jitter*h, (n_interior, 2))`` in row-major vertex
order while boundary vertices stay put, so periodic identification still holds.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

PERIODIC = 0
DIRICHLET = 1


def unit_square_mesh(m: int, jitter: float = 0.1, seed: int = 0):
    """Jittered m x m x 2 triangulation of [0,1]^2.

    Returns (xy float64 [(m+1)^2, 2], tri int32 [2 m^2, 3]); vertex (i, j) has index
    j*(m+1)+i (x index i, y index j); cell (i, j) gives triangles (a,b,c), (a,c,d) with
    a=(i,j), b=(i+1,j), c=(i+1,j+1), d=(i,j+1), both counter-clockwise.
    """
    h = 1.0 / m
    ii, jj = np.meshgrid(np.arange(m + 1), np.arange(m + 1), indexing="xy")
    xy = np.stack([ii.ravel() * h, jj.ravel() * h], axis=1).astype(np.float64)
    interior = np.flatnonzero((ii.ravel() > 0) & (ii.ravel() < m) & (jj.ravel() > 0) & (jj.ravel() < m))
    if jitter > 0 and interior.size:
        rng = np.random.default_rng(seed)
        xy[interior] += rng.uniform(-jitter * h, jitter * h, (interior.size, 2))
    ci, cj = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    ci = ci.ravel()
    cj = cj.ravel()
    a = cj * (m + 1) + ci
    b = a + 1
    c = a + (m + 1) + 1
    d = a + (m + 1)
    tri = np.empty((2 * m * m, 3), dtype=np.int32)
    tri[0::2] = np.stack([a, b, c], axis=1)
    tri[1::2] = np.stack([a, c, d], axis=1)
    return xy, tri


def centroids(xy, tri):
    return xy[tri].mean(axis=1)


def random_nodal(K: int, Np: int, seed: int):
    """Seeded standard-normal nodal field [K, Np] (float64)."""
    return np.random.default_rng(seed).standard_normal((K, Np))


# ----------------------------------------------------------------------------------
# Workload recipes
# ----------------------------------------------------------------------------------

@dataclass
class Forcing:
    """Separable forcing sum_m f_m(x, y) * tau_m(t), tau_m in {1, cos(w t), sin(w t)}."""
    funcs: List[Callable]  # f_m(x, y) -> array
    kinds: List[int]       # 0 const, 1 cos, 2 sin
    omegas: List[float]


TAU_CONST, TAU_COS, TAU_SIN = 0, 1, 2


def tau(kind: int, omega: float, t: float) -> float:
    if kind == TAU_CONST:
        return 1.0
    if kind == TAU_COS:
        return math.cos(omega * t)
    if kind == TAU_SIN:
        return math.sin(omega * t)
    raise ValueError(kind)


@dataclass
class Workload:
    name: str
    N: int
    m: int
    xy: np.ndarray
    tri: np.ndarray
    bc: int
    D_elem: np.ndarray
    v: tuple
    u0: Callable
    steps: int
    dt: Optional[float] = None          # None: derived from the stability bound
    dt_factor: float = 0.5               # fraction of the stability bound
    period: tuple = (1.0, 1.0)
    source: Optional[Forcing] = None
    ghost: Optional[Forcing] = None
    exact: Optional[Callable] = None     # u_e(x, y, t) when closed form known
    meta: dict = field(default_factory=dict)

    @property
    def K(self):
        return self.tri.shape[0]

    @property
    def Np(self):
        return (self.N + 1) * (self.N + 2) // 2


def heat_sin_mode(m: int = 16, N: int = 2, seed: int = 0, jitter: float = 0.1, steps: int = 200, D: float = 1.0):
    """Plain FP64 heat problem: u0 = sin(2 pi x) sin(2 pi y), periodic, D const, v = 0,
    dt = 0.1 h^2 / (D (N+1)^4).  Exact decay factor exp(-8 pi^2 D t)."""
    xy, tri = unit_square_mesh(m, jitter, seed)
    h = 1.0 / m
    dt = 0.1 * h * h / (D * (N + 1) ** 4)
    u0 = lambda x, y: np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    exact = lambda x, y, t: np.exp(-8 * np.pi ** 2 * D * t) * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    return Workload("heat_sin_N%d_m%d" % (N, m), N, m, xy, tri, PERIODIC, np.full(tri.shape[0], D),
                    (0.0, 0.0), u0, steps, dt=dt, exact=exact)


def circle_pulse(m: int = 256, N: int = 4, seed: int = 1, steps: int = 500, jitter: float = 0.1):
    """Convection-diffusion, v = (1, 0.5), D = 1 inside the circle r < 0.25 about (0.5, 0.5)
    (element centroid test) and 1e-4 outside, Gaussian pulse of width 0.05, periodic,
    dt = 0.5 x the stability bound."""
    xy, tri = unit_square_mesh(m, jitter, seed)
    cen = centroids(xy, tri)
    r = np.hypot(cen[:, 0] - 0.5, cen[:, 1] - 0.5)
    D = np.where(r < 0.25, 1.0, 1e-4)
    u0 = lambda x, y: np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2) / 0.05 ** 2)
    return Workload("circle_pulse_N%d_m%d" % (N, m), N, m, xy, tri, PERIODIC, D, (1.0, 0.5), u0, steps,
                    dt=None, dt_factor=0.5)


def manufactured_dirichlet(m: int, N: int = 3, seed: int = 10, D: float = 1.0, T: float = 2.0 ** -10,
                           jitter: float = 0.1):
    """u = sin(pi x) sin(pi y) cos t with source s = sin sin (-sin t + 2 pi^2 D cos t),
    v = 0, Dirichlet data from the exact solution."""
    xy, tri = unit_square_mesh(m, jitter, seed)
    ss = lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
    src = Forcing([lambda x, y: -ss(x, y), lambda x, y: 2 * np.pi ** 2 * D * ss(x, y)], [TAU_SIN, TAU_COS], [1.0, 1.0])
    ghost = Forcing([ss], [TAU_COS], [1.0])
    exact = lambda x, y, t: ss(x, y) * np.cos(t)
    return Workload("mms_dirichlet_N%d_m%d" % (N, m), N, m, xy, tri, DIRICHLET, np.full(tri.shape[0], D),
                    (0.0, 0.0), lambda x, y: ss(x, y), steps=0, dt=None, dt_factor=0.5,
                    source=src, ghost=ghost, exact=exact, meta={"T": T})


def gaussian_exact(x0, y0, a=(0.0, 0.0), D=1.0, D0=2.0, M=1.0, period=(10.0, 10.0), images=2):
    """Mass M loaded at (x0, y0) at t = -D0/D, diffusing with D and carried by a, on the
    periodic domain: the free-space solution M/(4 pi (D t + D0)) exp(-|x - x0 - a t|^2 /
    (4 (D t + D0))) summed over the periodic images within `images` periods (the next ones
    are below 1e-25 for the paper's D0 = 2 and a 10-wide domain)."""
    def f(x, y, t):
        s = D * t + D0
        out = np.zeros(np.broadcast(x, y).shape)
        cx, cy = x0 + a[0] * t, y0 + a[1] * t
        for i in range(-images, images + 1):
            for j in range(-images, images + 1):
                dx = x - cx - i * period[0]
                dy = y - cy - j * period[1]
                out = out + np.exp(-(dx * dx + dy * dy) / (4 * s))
        return M / (4 * np.pi * s) * out
    return f


def paper_gaussian(m: int, N: int, advection: bool = False, jitter: float = 0.0, seed: int = 0, T: float = 0.5):
    """The paper's verification problems (Sec. 5.1 diffusion, Sec. 5.2 advection-diffusion),
    on stand-ins for its grid a: the 10 x 10 square [0, 10] x [-5, 5] cut into m x m cells
    split by "/" diagonals (each triangle pair a parallelogram, as in grid a; jitter > 0
    moves interior vertices so the reconstruction truncates areas, in the spirit of grids
    b and c), periodic, D = 1, D0 = 2, M = 1; diffusion: (x0, y0) = (5, 0), a = 0;
    advection-diffusion: (x0, y0) = (4, -1), a = (6, 6).  Final time 0.5."""
    xy, tri = unit_square_mesh(m, jitter, seed)
    xy = xy * 10.0
    xy[:, 1] -= 5.0
    if advection:
        x0, y0, a = 4.0, -1.0, (6.0, 6.0)
    else:
        x0, y0, a = 5.0, 0.0, (0.0, 0.0)
    exact = gaussian_exact(x0, y0, a)
    return Workload("%s_N%d_m%d" % ("advdiff" if advection else "diffusion", N, m), N, m, xy, tri, PERIODIC,
                    np.ones(tri.shape[0]), a, lambda x, y: exact(x, y, 0.0), steps=0, period=(10.0, 10.0),
                    exact=exact, meta={"T": T})


def fourier_u0(seed: int, kmax: int = 3):
    """Random low-mode periodic field sum_{|kx|,|ky|<=kmax} a_k {sin,cos}, a_k ~ N(0,1)/(1+|k|^2)."""
    rng = np.random.default_rng(seed)
    terms = []
    for kx in range(-kmax, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            w = 1.0 / (1.0 + kx * kx + ky * ky)
            terms.append((kx, ky, rng.standard_normal() * w, rng.standard_normal() * w))

    def f(x, y):
        out = np.zeros_like(x, dtype=np.float64)
        for kx, ky, a, b in terms:
            ph = 2 * np.pi * (kx * x + ky * y)
            out += a * np.cos(ph) + b * np.sin(ph)
        return out
    return f


def batched_heat(seed: int = 2, nprob: int = 64, side_lo: int = 8, side_hi: int = 256, steps: int = 100,
                 N_lo: int = 1, N_hi: int = 6):
    """Independent periodic heat problems with random mesh side, order, D and Fourier u0."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(nprob):
        m = int(rng.integers(side_lo, side_hi + 1))
        N = int(rng.integers(N_lo, N_hi + 1))
        D = float(np.exp(rng.uniform(np.log(1e-3), np.log(1.0))))
        mesh_seed = int(rng.integers(0, 2 ** 31 - 1))
        u_seed = int(rng.integers(0, 2 ** 31 - 1))
        xy, tri = unit_square_mesh(m, 0.1, mesh_seed)
        out.append(Workload("batch%d_N%d_m%d" % (p, N, m), N, m, xy, tri, PERIODIC, np.full(tri.shape[0], D),
                            (0.0, 0.0), fourier_u0(u_seed), steps, dt=None, dt_factor=0.5))
    return out


def _circle_mesh(m, mesh_seed, cx, cy, rad, inside_high, contrast):
    xy, tri = unit_square_mesh(m, 0.1, mesh_seed)
    cen = centroids(xy, tri)
    ins = np.hypot(cen[:, 0] - cx, cen[:, 1] - cy) < rad
    D = np.where(ins == inside_high, 1.0, 1.0 / contrast)
    return xy, tri, D


@dataclass
class Request:
    rid: int
    arrival: float
    workload: Workload
    fp64_check: bool


def serve_stream(seed: int = 3, nreq: int = 2000, rate: float = 200.0, K_lo: float = 1e3, K_hi: float = 1e6,
                 N_lo: int = 2, N_hi: int = 6, steps_lo: int = 50, steps_hi: int = 500, check_frac: float = 0.01,
                 build_mesh: bool = True):
    """Poisson stream of solve requests: jittered meshes of log-uniform size, random order,
    piecewise-constant D across a random circle, random velocity and step count."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(nreq):
        t += rng.exponential(1.0 / rate)
        K = float(np.exp(rng.uniform(np.log(K_lo), np.log(K_hi))))
        m = max(2, int(round(math.sqrt(K / 2.0))))
        N = int(rng.integers(N_lo, N_hi + 1))
        contrast = float(np.exp(rng.uniform(0.0, np.log(1e4))))
        cx, cy = rng.uniform(0.25, 0.75, 2)
        rad = float(rng.uniform(0.1, 0.3))
        inside_high = bool(rng.integers(0, 2))
        vx, vy = rng.uniform(-1.0, 1.0, 2)
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        mesh_seed = int(rng.integers(0, 2 ** 31 - 1))
        check = bool(rng.uniform() < check_frac)
        build = (lambda mm, ms, ccx, ccy, rr, ih, con: (lambda: _circle_mesh(mm, ms, ccx, ccy, rr, ih, con)))(
            m, mesh_seed, cx, cy, rad, inside_high, contrast)
        if build_mesh:
            xy, tri, D = build()
        else:
            xy = tri = D = None
        w0 = 0.05 + 0.1 * rng.uniform()
        u0 = (lambda ccx, ccy, ww: (lambda x, y: np.exp(-((x - ccx) ** 2 + (y - ccy) ** 2) / ww ** 2)))(cx, cy, w0)
        wl = Workload("req%d_N%d_m%d" % (i, N, m), N, m, xy, tri, PERIODIC, D, (float(vx), float(vy)), u0, steps,
                      dt=None, dt_factor=0.5, meta={"mesh_seed": mesh_seed, "contrast": contrast, "build": build,
                                                    "triangles": 2 * m * m})
        reqs.append(Request(i, t, wl, check))
    return reqs
