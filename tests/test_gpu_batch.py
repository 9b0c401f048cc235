"""Batched stepping (rdg_batch_*): members of different orders, sizes, precisions and
boundary conditions advanced together by one CUDA graph give the same states as each
problem stepped alone, and a small FP64 member follows the oracle.

Equality with the lone solve is bitwise for members without time-dependent forcing (the
same kernels with the same arguments run in both) and to rounding of the stage time
(t0 + (n + off) dt summed in another order) for forced members.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1912_06221_gb300 as rdg
from synth import unit_square_mesh, random_nodal, PERIODIC, DIRICHLET
from oracle.mesh import Mesh
from oracle.rhs import Problem, stable_dt


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - b) / max(np.linalg.norm(b), 1e-300))


# (N, m, precision, bc, velocity, forced)
MEMBERS = [(1, 11, rdg.FP32, PERIODIC, (0.0, 0.0), False),
           (2, 4, rdg.FP64, PERIODIC, (0.5, 0.25), False),
           (3, 9, rdg.FP32, DIRICHLET, (0.0, 0.0), True),
           (4, 6, rdg.FP64, PERIODIC, (-0.3, 0.8), False),
           (5, 13, rdg.FP32, PERIODIC, (1.0, 0.5), False),
           (6, 5, rdg.FP64, DIRICHLET, (0.2, 0.0), True),
           (6, 7, rdg.FP32, PERIODIC, (0.4, -0.2), False)]


def _member(i, N, m, prec, bc, v, forced):
    xy, tri = unit_square_mesh(m, 0.1, 20 + i)
    K = tri.shape[0]
    D = np.where(np.random.default_rng(i).uniform(size=K) < 0.4, 1.0, 0.05)
    s = rdg.Solver(xy, tri, N, D, v=v, bc=bc, precision=prec)
    if forced:
        xyn = s.node_coords()
        src = [(np.sin(3 * xyn[..., 0]) * xyn[..., 1], rdg.TAU_COS, 2.0)]
        gh = []
        if s.B:
            g = s.ghost_coords()
            gh = [(g[..., 0] - g[..., 1], rdg.TAU_SIN, 1.0)]
        s.set_forcing(src, gh)
    u0 = np.ascontiguousarray(random_nodal(s.K, s.Np, 40 + i) * 0.1 + 1.0, dtype=s.np_dtype)
    s.set_state(u0)
    h = 1.0 / m
    dt = 0.05 * h * h / (N + 1) ** 4
    return s, u0, dt, xy, tri, D


def _build(members):
    out = []
    for i, spec in enumerate(members):
        a = _member(i, *spec)
        b = _member(i, *spec)      # the same problem, stepped alone
        out.append((spec, a, b))
    return out


def _check(items, t_alone, nsteps):
    for (spec, a, b) in items:
        sa, _, dt = a[0], a[1], a[2]
        sb = b[0]
        sb.solve_to_time(t_alone, dt, nsteps)
        ga, gb = sa.get_state_host(), sb.get_state_host()
        forced = spec[5]
        if forced:
            tol = 1e-13 if spec[2] == rdg.FP64 else 1e-6
            assert relerr(ga, gb) < tol, spec
        else:
            assert np.array_equal(ga, gb), spec


def test_batch_equals_alone_and_membership_changes():
    items = _build(MEMBERS)
    bt = rdg.Batch(chunk=16)
    for (spec, a, b) in items:
        bt.add(a[0], a[2], t0=0.0)
    assert len(bt) == len(MEMBERS)
    bt.step(37)                          # two graph replays and five direct steps
    bt.synchronize()
    _check(items, 0.0, 37)
    # drop a member, add it back at its current time, step again (graph re-captured)
    spec, a, b = items[3]
    bt.remove(a[0])
    assert len(bt) == len(MEMBERS) - 1
    bt.step(16)
    bt.synchronize()
    for j, (sp, aa, bb) in enumerate(items):
        if j != 3:
            bb[0].solve_to_time(37 * aa[2], aa[2], 16)
    for j, (sp, aa, bb) in enumerate(items):
        if j == 3:
            continue
        ga, gb = aa[0].get_state_host(), bb[0].get_state_host()
        if sp[5]:
            assert relerr(ga, gb) < (1e-13 if sp[2] == rdg.FP64 else 1e-6)
        else:
            assert np.array_equal(ga, gb)
    assert np.array_equal(a[0].get_state_host(), b[0].get_state_host())   # untouched while removed
    bt.add(a[0], a[2], t0=37 * a[2])
    bt.step(3)
    bt.synchronize()
    b[0].solve_to_time(37 * a[2], a[2], 3)
    assert np.array_equal(a[0].get_state_host(), b[0].get_state_host())
    bt.close()
    for (spec, a, b) in items:
        a[0].close()
        b[0].close()


def test_batch_member_follows_oracle():
    """A FP64 member (N=2, Dirichlet, forcing) stepped inside a batch with an FP32 N=5
    problem follows the oracle's SSP-RK3 steps."""
    N, m = 2, 5
    xy, tri = unit_square_mesh(m, 0.1, 7)
    K = tri.shape[0]
    D = np.where(np.random.default_rng(1).uniform(size=K) < 0.5, 1.0, 0.1)
    v = (0.6, -0.3)
    s = rdg.Solver(xy, tri, N, D, v=v, bc=DIRICHLET, precision=rdg.FP64)
    me = Mesh(xy, tri, N, bc=DIRICHLET)
    xyn = s.node_coords()
    s.set_forcing([(np.cos(2 * xyn[..., 0]), rdg.TAU_SIN, 3.0)],
                  [(s.ghost_coords()[..., 0] ** 2, rdg.TAU_CONST, 0.0)])
    pr = Problem(me, D, v=v, source=[(np.cos(2 * me.x), rdg.TAU_SIN, 3.0)],
                 ghost_fn=lambda x, y, t: x * x)
    u0 = random_nodal(K, s.Np, 9) * 0.1 + me.y
    dt = stable_dt(pr, 0.4, 20)
    other, _, dto, _, _, _ = _member(0, 5, 13, rdg.FP32, PERIODIC, (1.0, 0.5), False)
    s.set_state(u0)
    t0 = 0.25
    bt = rdg.Batch(chunk=8)
    bt.add(other, dto)
    bt.add(s, dt, t0=t0)
    bt.step(19)
    bt.synchronize()
    want = pr.solve(u0, t0, dt, 19)
    assert relerr(s.get_state_host(), want) < 1e-10
    bt.close()
    s.close()
    other.close()


def test_batch_errors():
    s, _, dt, _, _, _ = _member(0, 2, 4, rdg.FP64, PERIODIC, (0.0, 0.0), False)
    bt = rdg.Batch()
    bt.step(5)                           # empty batch: nothing to do
    bt.add(s, dt)
    with pytest.raises(rdg.RdgError) as e:
        bt.add(s, dt)
    assert e.value.code == rdg.rdg.RDG_EINVAL
    with pytest.raises(rdg.RdgError):
        bt.step(-1)
    s2, _, _, _, _, _ = _member(1, 1, 3, rdg.FP32, PERIODIC, (0.0, 0.0), False)
    with pytest.raises(rdg.RdgError):
        bt.add(s2, 0.0)
    with pytest.raises(rdg.RdgError):
        bt.remove(s2)
    bt.step(0)
    bt.synchronize()
    bt.close()
    s.close()
    s2.close()


def test_batch_chunk_change_keeps_results():
    """Replaying the same steps with another graph chunk gives the same states bit for bit."""
    items = _build(MEMBERS[:3])
    bt = rdg.Batch(chunk=16)
    for (spec, a, b) in items:
        bt.add(a[0], a[2])
    bt.step(20)
    bt.synchronize()
    got = [a[0].get_state_host() for (_, a, _) in items]
    for (spec, a, b) in items:
        a[0].set_state(a[1])
    bt.set_chunk(7)
    with pytest.raises(rdg.RdgError):
        bt.set_chunk(0)
    bt2 = rdg.Batch(chunk=7)
    for (spec, a, b) in items:
        bt.remove(a[0])
        bt2.add(a[0], a[2])
    bt2.step(20)
    bt2.synchronize()
    for g, (spec, a, b) in zip(got, items):
        if spec[5]:
            assert relerr(a[0].get_state_host(), g) < (1e-13 if spec[2] == rdg.FP64 else 1e-6)
        else:
            assert np.array_equal(a[0].get_state_host(), g)
    bt.close()
    bt2.close()
    for (spec, a, b) in items:
        a[0].close()
        b[0].close()


def test_autotune_picks_a_valid_form_and_caches():
    from paper_1912_06221_gb300 import autotune
    xy, tri = unit_square_mesh(12, 0.1, 1)
    D = np.full(tri.shape[0], 0.3)
    c1 = autotune.choose_precision(xy, tri, 3, D)
    assert c1["precision"] in (rdg.FP32, rdg.FP32_3XTF32) and not c1["cached"]
    assert set(c1["ms"]) == {"fp32", "fp32_3xtf32"} and all(t > 0 for t in c1["ms"].values())
    c2 = autotune.choose_precision(xy, tri, 3, D)
    assert c2["cached"] and c2["precision"] == c1["precision"]
    c6 = autotune.choose_precision(xy, tri, 6, D)
    assert c6["precision"] == rdg.FP32 and set(c6["ms"]) == {"fp32"}


def test_batch_member_with_lsrk_integrator_equals_alone():
    """A member stepped with the paper's low-storage scheme inside a batch (beside an
    SSP-RK3 member) ends where the same solve alone does."""
    specs = [(4, 6, rdg.FP32, PERIODIC, (0.4, 0.2), False), (2, 5, rdg.FP64, PERIODIC, (0.0, 0.0), False)]
    items = _build(specs)
    (_, a0, b0), (_, a1, b1) = items
    a0[0].set_integrator(rdg.LSRK54)
    b0[0].set_integrator(rdg.LSRK54)
    bt = rdg.Batch(chunk=8)
    bt.add(a0[0], a0[2])
    bt.add(a1[0], a1[2])
    bt.step(19)
    bt.synchronize()
    b0[0].solve_to_time(0.0, a0[2], 19)
    b1[0].solve_to_time(0.0, a1[2], 19)
    assert np.array_equal(a0[0].get_state_host(), b0[0].get_state_host())
    assert np.array_equal(a1[0].get_state_host(), b1[0].get_state_host())
    bt.close()
    for (_, a, b) in items:
        a[0].close()
        b[0].close()
