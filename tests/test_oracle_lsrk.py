"""Pins of the oracle's five-stage fourth-order low-storage Runge-Kutta step (the paper's
integrator, Sec. 5) by what a fourth-order scheme must satisfy:

* for u' = z u its one-step factor agrees with e^z up to z^4: the local error falls by
  2^5 when z is halved;
* it integrates u' = p(t) exactly for polynomials p of degree <= 3 (stage times c_i);
* over many steps the global error of u' = z u falls by 2^4 when dt is halved.
"""
import math

import numpy as np

from oracle.rhs import Problem


class _Scalar:
    """A stand-in for Problem with rhs = lam * u + p(t)."""

    def __init__(self, lam, p=lambda t: 0.0):
        self.lam, self.p = lam, p

    def rhs(self, u, t=0.0):
        return self.lam * u + self.p(t)


def _step(prob, u, t, dt):
    return Problem.lsrk_step(prob, np.array([u], float), t, dt)[0]


def test_lsrk_local_error_is_fifth_order():
    errs = []
    for z in (0.2, 0.1, 0.05):
        errs.append(abs(_step(_Scalar(z), 1.0, 0.0, 1.0) - math.exp(z)))
    assert 28 < errs[0] / errs[1] < 36 and 28 < errs[1] / errs[2] < 36, errs


def test_lsrk_integrates_cubics_in_time_exactly():
    t0, dt = 0.3, 0.7
    p = lambda t: 1.0 - 2.0 * t + 3.0 * t ** 2 + 5.0 * t ** 3
    P = lambda t: t - t ** 2 + t ** 3 + 1.25 * t ** 4
    got = _step(_Scalar(0.0, p), 2.0, t0, dt)
    assert abs(got - (2.0 + P(t0 + dt) - P(t0))) < 1e-13


def test_lsrk_global_error_fourth_order():
    lam, T = -1.3, 1.0
    errs = []
    for n in (8, 16, 32):
        u = np.array([1.0])
        for k in range(n):
            u = Problem.lsrk_step(_Scalar(lam), u, k * T / n, T / n)
        errs.append(abs(u[0] - math.exp(lam * T)))
    assert 14 < errs[0] / errs[1] < 18 and 14 < errs[1] / errs[2] < 18, errs
