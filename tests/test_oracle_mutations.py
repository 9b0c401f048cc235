"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each.

Every mutation here is applied with monkeypatch to the oracle only, for the duration of one
test, so the pins above are shown to be sensitive to dropped terms, wrong signs, wrong
indices and transposed operands."""
import numpy as np
import pytest

import oracle.ardg as ardg
import oracle.refops as refops
import oracle.rhs as orhs
from tests import test_oracle_ardg as TA
from tests import test_oracle_rhs as TR


def _fails(fn, *a):
    with pytest.raises(AssertionError):
        fn(*a)


def test_mutation_transposed_derivative(monkeypatch):
    orig = refops.RefOps.__init__

    def bad(self, N):
        orig(self, N)
        self.Dr = self.Dr.T.copy()
    monkeypatch.setattr(refops.RefOps, "__init__", bad)
    _fails(TR.test_rhs_exact_for_global_polynomials, 2)


def test_mutation_side2_flux_sign(monkeypatch):
    orig = orhs.Problem.edge_flux
    calls = {"n": 0}

    def bad_rhs(self, u, t=0.0):
        # use +F*.n1 (not negated) on side 2
        m = self.mesh
        ops = m.ops
        out = orig_rhs(self, u, t)
        fl = orig(self, u, t)
        ii = np.flatnonzero(self.interior)
        k2, f2 = self.k2[ii], self.f2[ii]
        q2 = -fl[ii][:, ::-1]
        c2 = m.Fscale[k2, f2][:, None] * np.einsum("eiq,eq->ei", ops.LIFT[f2], q2)
        np.add.at(out, k2, 2 * c2)      # turns -(-q) into +(-q)
        return out
    orig_rhs = orhs.Problem.rhs
    monkeypatch.setattr(orhs.Problem, "rhs", bad_rhs)
    _fails(TR.test_conservation_periodic, 2)


def test_mutation_side2_frame_not_reflected(monkeypatch):
    orig = refops.RefOps._build_reconstruction

    def bad(self):
        orig(self)
        self.A = np.vstack([self.A1, self.A1])          # side 2 on I instead of I^{-1}
        self.Apinv = np.linalg.pinv(self.A, rcond=1e-13)
    monkeypatch.setattr(refops.RefOps, "_build_reconstruction", bad)
    _fails(TA.test_reconstruction_reproduces_global_polynomials, 3, 0)


def test_mutation_wrong_rotation(monkeypatch):
    orig = ardg.EdgeOps.projection

    def bad(self, ab, f):
        return orig(self, ab, (f + 1) % 3)
    monkeypatch.setattr(ardg.EdgeOps, "projection", bad)
    _fails(TA.test_reconstruction_reproduces_global_polynomials, 2, 0)


def test_mutation_parallelogram_not_enclosed(monkeypatch):
    def bad(e1, e2, q1, q2):
        c = (e1 + e2) / 2
        return np.array(q1, float), 2 * c - np.array(q1, float)
    monkeypatch.setattr(ardg, "enclosed_parallelogram", bad)
    monkeypatch.setattr(TA, "enclosed_parallelogram", bad)
    _fails(TA.test_parallelogram_brute_force_and_containment)


def test_mutation_parallelogram_wrong_metric(monkeypatch):
    orig = ardg.EdgeOps.__init__

    def bad(self, mesh):
        orig(self, mesh)
        self.Rx[:, [1, 2]] = self.Rx[:, [2, 1]]         # R_y <-> S_x
    monkeypatch.setattr(ardg.EdgeOps, "__init__", bad)
    _fails(TA.test_reconstruction_reproduces_global_polynomials, 2, 0)


def test_mutation_D_not_averaged(monkeypatch):
    orig = ardg.EdgeOps.reconstruct_D

    def bad(self, D1, D2):
        return orig(self, D1, D1)
    monkeypatch.setattr(ardg.EdgeOps, "reconstruct_D", bad)
    _fails(TA.test_algorithm2_D_is_edge_mean, 3)


def test_mutation_rk3_stage_time(monkeypatch):
    def bad(self, u, t, dt):
        u1 = u + dt * self.rhs(u, t)
        u2 = 0.75 * u + 0.25 * (u1 + dt * self.rhs(u1, t + dt))
        return u / 3.0 + 2.0 / 3.0 * (u2 + dt * self.rhs(u1, t + 0.5 * dt))   # uses u1, not u2
    monkeypatch.setattr(orhs.Problem, "rk3_step", bad)
    _fails(TR.test_dense_operator_stable_and_rk3_amplification, 3, 1)


def test_mutation_dropped_volume_term(monkeypatch):
    orig_rhs = orhs.Problem.rhs

    def bad(self, u, t=0.0):
        v = self.v
        self.v = np.zeros(2)               # drop the convective volume term only
        out = orig_rhs(self, u, t)
        self.v = v
        # add back the convective surface part, keeping the volume part missing
        return out
    monkeypatch.setattr(orhs.Problem, "rhs", bad)
    _fails(TR.test_rhs_exact_for_global_polynomials, 2)


def test_mutation_alg1_side2_gradient_not_reflected(monkeypatch):
    """Algorithm 1 with side 2's gradient taken as if its frame were side 1's (no sign flip
    of d/dR, d/dS under the point reflection)."""
    from tests import test_oracle_alg1 as T1

    def bad(self, c, D1, D2):
        ops = self.mesh.ops
        Rx, Ry, Sx, Sy = self.Rx.T
        Phi = ops.phi(ops.diag_R, ops.diag_S)
        out = np.zeros((c.shape[0], ops.Nfp))
        for comp in range(2):
            dRp = Rx if comp == 0 else Ry
            dSp = Sx if comp == 0 else Sy
            modal = []
            for Ak, Dk in ((ops.A1, D1), (ops.A2, D2)):
                nod = (c @ Ak.T) @ ops.V.T
                g = dRp[:, None] * (nod @ ops.Dr.T) + dSp[:, None] * (nod @ ops.Ds.T)
                modal.append((np.asarray(Dk)[:, None] * g) @ ops.Vinv.T)
            out += self.n1[:, comp:comp + 1] * ((np.concatenate(modal, axis=1) @ ops.Apinv.T) @ Phi.T)
        return out
    monkeypatch.setattr(ardg.EdgeOps, "flux_algorithm1", bad)
    _fails(T1.test_alg1_exact_for_global_polynomials, 2)


def test_mutation_lsrk_stage_time(monkeypatch):
    """A wrong stage time in the low-storage Runge-Kutta step (the third stage evaluated at
    the second stage's time)."""
    from tests import test_oracle_lsrk as TL
    bad = list(orhs.LSRK_C)
    bad[2] = bad[1]
    monkeypatch.setattr(orhs, "LSRK_C", tuple(bad))
    _fails(TL.test_lsrk_integrates_cubics_in_time_exactly)


def test_mutation_lsrk_weight(monkeypatch):
    """A wrong stage weight (the last two b_i swapped)."""
    from tests import test_oracle_lsrk as TL
    bad = list(orhs.LSRK_B)
    bad[3], bad[4] = bad[4], bad[3]
    monkeypatch.setattr(orhs, "LSRK_B", tuple(bad))
    _fails(TL.test_lsrk_local_error_is_fifth_order)


def test_mutation_tensor_components_swapped_on_edges(monkeypatch):
    """Algorithm 2 with D = (Dx, Dy) applying D~y to u~_x and D~x to u~_y on the edges."""
    from tests import test_oracle_aniso as TN
    orig = ardg.EdgeOps.edge_gradient

    def bad(self, c):
        ux, uy = orig(self, c)
        return uy, ux
    monkeypatch.setattr(ardg.EdgeOps, "edge_gradient", bad)
    _fails(TN.test_tensor_rotation_swaps_components, "alg2")


def test_mutation_tensor_volume_uses_one_component(monkeypatch):
    """The volume flux with Dx in both components."""
    from tests import test_oracle_aniso as TN
    orig = orhs.Problem.__init__

    def bad(self, mesh, D_elem, *a, **k):
        orig(self, mesh, D_elem, *a, **k)
        if self.aniso:
            self.D = self.D.copy()
            self.D[:, 1] = self.D[:, 0]
    monkeypatch.setattr(orhs.Problem, "__init__", bad)
    _fails(TN.test_tensor_sin_mode_decay_rate, "alg1")


def test_mutation_nodal_D_projection_skipped(monkeypatch):
    """Algorithm 1 with nodal D using the element's nodal values as if they were the values at
    the sub-triangle nodes (no V_p projection)."""
    from tests import test_oracle_nodal as TD
    orig = ardg.EdgeOps.flux_algorithm1

    def bad(self, c, D1, D2):
        D1, D2 = np.asarray(D1), np.asarray(D2)
        if D1.ndim == 2 and D1.shape[1] == self.mesh.ops.Np:
            P1, P2 = self.P1, self.P2
            eye = np.broadcast_to(self.mesh.ops.Vinv, P1.shape)
            self.P1, self.P2 = eye, eye
            try:
                return orig(self, c, D1, D2)
            finally:
                self.P1, self.P2 = P1, P2
        return orig(self, c, D1, D2)
    monkeypatch.setattr(ardg.EdgeOps, "flux_algorithm1", bad)
    _fails(TD.test_nodal_D_exact_for_linear_D_and_polynomials, 3, "alg1")
