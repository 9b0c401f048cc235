"""The oracle on sampled patches (oracle/patch.py) against the oracle on the whole mesh.

The patch helper lets the oracle check single elements of meshes far too large for it (the
131072-triangle circle pulse).  It is pinned here against the full-mesh oracle on small
periodic meshes: one ring of neighbours reproduces the right-hand side on the sampled
elements, three rings reproduce an SSP-RK3 step, and two rings do not (so the sampled rows
really depend on the third ring, which is what makes the comparison meaningful)."""
import numpy as np
import pytest

from synth import random_nodal, unit_square_mesh
from oracle.mesh import Mesh
from oracle.patch import PatchProblem, face_neighbours
from oracle.rhs import Problem


def _case(m=6, N=3, seed=3, iface="alg1"):
    xy, tri = unit_square_mesh(m, 0.1, seed)
    K = tri.shape[0]
    D = np.where(np.arange(K) % 3 == 0, 1.0, 0.05)
    pr = Problem(Mesh(xy, tri, N), D, v=(0.7, -0.4), interface=iface)
    return xy, tri, K, D, pr


@pytest.mark.parametrize("iface", ["alg1", "alg2"])
def test_patch_rhs_equals_full_mesh_rhs(iface):
    xy, tri, K, D, pr = _case(iface=iface)
    u = random_nodal(K, pr.mesh.ops.Np, 1)
    ref = pr.rhs(u, 0.3)
    # corners and sides of the periodic square (wrap-around faces) and interior elements
    sample = [0, 1, 5, 11, 30, 41, 70, K - 1]
    pp = PatchProblem(xy, tri, 3, D, sample, v=(0.7, -0.4), rings=1, interface=iface)
    got = pp.rhs(u, 0.3)
    assert np.abs(got - ref[sample]).max() < 1e-13 * np.abs(ref).max()
    assert pp.patch_elements < K


def test_patch_rk3_step_needs_three_rings():
    xy, tri, K, D, pr = _case()
    u = random_nodal(K, pr.mesh.ops.Np, 2)
    ref = pr.rk3_step(u, 0.0, 2e-3)
    sample = [3, 17, 40]
    scale = np.abs(ref).max()
    p3 = PatchProblem(xy, tri, 3, D, sample, v=(0.7, -0.4), rings=3, interface="alg1")
    assert np.abs(p3.rk3_step(u, 0.0, 2e-3) - ref[sample]).max() < 1e-13 * scale
    p2 = PatchProblem(xy, tri, 3, D, sample, v=(0.7, -0.4), rings=2, interface="alg1")
    assert np.abs(p2.rk3_step(u, 0.0, 2e-3) - ref[sample]).max() > 1e-6 * scale


def test_face_neighbours_periodic_shifts():
    xy, tri = unit_square_mesh(4, 0.1, 1)
    nk, sh = face_neighbours(xy, tri)
    K = tri.shape[0]
    assert (nk >= 0).all()
    # the relation is symmetric and shifts are whole periods that cancel
    for k in range(K):
        for f in range(3):
            n = nk[k, f]
            back = [g for g in range(3) if nk[n, g] == k and np.allclose(sh[n, g], -sh[k, f])]
            assert back, (k, f)
            assert np.all(np.isin(sh[k, f], (-1.0, 0.0, 1.0)))
    with pytest.raises(ValueError):
        PatchProblem(xy, tri, 2, 1.0, [0, 0])
