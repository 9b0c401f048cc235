"""The GEMM form of the per-edge diffusive operator (host reference factors of the library,
no GPU): for every edge of jittered periodic and Dirichlet meshes and both sides,

    sum_rho kappa_rho sum_m psi_m(alpha_k, beta_k) X[k][m][., rho, perm_f(.)]

equals the oracle's (kappa_R D_R + kappa_S D_S) A^+_k P_k (Sec. 4.4-4.5, Eq. totalProjection),
where (alpha_k, beta_k) is the parallelogram apex in side k's rotated frame and
kappa = n1 . (R_x, R_y), n1 . (S_x, S_y).  The oracle builds P_k = V^{-1} V_p V_rf^{-1} by
evaluating the basis at the mapped nodes; the library expands V_p in the apex coordinates
once per order, so the two routes are independent.
"""
import numpy as np
import pytest

import paper_1912_06221_gb300 as rdg
from synth import unit_square_mesh, PERIODIC, DIRICHLET
from oracle.mesh import Mesh
from oracle.ardg import EdgeOps
from oracle.refops import psi


def _lib_or_skip():
    try:
        rdg.load()
    except RuntimeError as e:
        pytest.skip(str(e))


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("bc", [PERIODIC, DIRICHLET])
def test_gemm_form_matches_oracle_projection(N, bc):
    _lib_or_skip()
    Np, Nfp = rdg.np_of(N), N + 1
    X = rdg.reference_operator(N, 6).reshape(2, Np, Nfp, 2, Np)
    perm = rdg.reference_operator(N, 7).reshape(3, Np).astype(int)
    xy, tri = unit_square_mesh(4, 0.2, 11)
    me = Mesh(xy, tri, N, bc=bc)
    eo = EdgeOps(me)
    ops = me.ops
    worst = 0.0
    for e, (k1, f1, k2, f2, _, _) in enumerate(me.edges):
        Rx, Ry, Sx, Sy = eo.Rx[e]
        n = eo.n1[e]
        kap = np.array([n[0] * Rx + n[1] * Ry, n[0] * Sx + n[1] * Sy])
        K = kap[0] * ops.DR + kap[1] * ops.DS              # [Nfp][Mp]
        for side, (ab, P, f) in enumerate(((eo.ab1[e], eo.P1[e], f1), (eo.ab2[e], eo.P2[e], f2 if k2 >= 0 else 1))):
            want = K @ ops.Apinv[:, side * Np:(side + 1) * Np] @ P
            ph = psi(N, ab[0], ab[1])[0]                   # [Np]
            G = np.einsum("m,r,mirl->il", ph, kap, X[side])  # rotated node order
            got = G[:, perm[f]]                            # natural node order
            scale = np.abs(want).max()
            worst = max(worst, np.abs(got - want).max() / scale)
    assert worst < 1e-11, worst


@pytest.mark.parametrize("N", [1, 3, 6])
def test_rotated_face_nodes(N):
    """The shared face's nodes sit at the same rotated indices for every face f."""
    _lib_or_skip()
    Np, Nfp = rdg.np_of(N), N + 1
    perm = rdg.reference_operator(N, 7).reshape(3, Np).astype(int)
    hyp = rdg.reference_operator(N, 8).astype(int)
    assert hyp.shape == (Nfp,)
    from oracle.refops import RefOps
    ops = RefOps(N)
    for f in range(3):
        assert list(perm[f][ops.Fmask[f]]) == list(hyp)
