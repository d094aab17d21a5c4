"""FP64 reference of the Chebyshev window propagator (test infrastructure).

A window of n_w explicit substeps of Eq. HeatTransport (pair-flux part,
d theta_i/dt = K F_i(theta)), tau = n_w dt, is advanced by s stages of the
first-order damped Chebyshev recurrence (the RKC family of Verwer, Hundsdorfer
and Sommeijer): with w0 = 1 + eps/s^2, w1 = T_s(w0)/T_s'(w0), b_j = 1/T_j(w0),

  Y_0 = theta,   Y_1 = Y_0 + (w1/w0) tau K F(Y_0),
  Y_j = mu_j Y_{j-1} + nu_j Y_{j-2} + mut_j tau K F(Y_{j-1}),   j = 2..s
      (evaluated as Y_{j-1} + nu_j (Y_{j-2} - Y_{j-1}) + ..., since mu_j + nu_j = 1),
  mu_j = 2 w0 b_j / b_{j-1},  nu_j = -b_j / b_{j-2},  mut_j = 2 w1 b_j / b_{j-1},

so that on a linear mode (K F = -lambda theta) Y_s = P_s(-tau lambda) theta with
P_s(z) = T_s(w0 + w1 z) / T_s(w0): P_s(0) = 1, P_s'(0) = 1, |P_s| <= 1 on
[-beta, 0], beta = (1 + w0) / w1 (about (2 - 4 eps / 3) s^2).  Every stage is an
affine combination (mu_j + nu_j = 1) of states plus a conservative flux, so the
sum of theta is kept.  T_j are Chebyshev polynomials of the first kind.

The second-order member of the family (coefficients2, window2) matches the
exponential to second order at z = 0; it needs about 1.5 times the stages for
the same stability interval.

Pinned in tests/test_oracle_window.py against the closed forms
T_s(x) = cos(s arccos x) / cosh(s arccosh x), a linear-regime lattice mode,
conservation and the uniform fixed point.
"""
from __future__ import annotations

import math

import numpy as np

from . import flux_sum


def cheb(j: int, x: float) -> float:
    """T_j(x) by the three-term recurrence."""
    t0, t1 = 1.0, x
    if j == 0:
        return t0
    for _ in range(j - 1):
        t0, t1 = t1, 2.0 * x * t1 - t0
    return t1


def dcheb(j: int, x: float) -> float:
    """T_j'(x) by differentiating the recurrence."""
    t0, t1 = 1.0, x
    d0, d1 = 0.0, 1.0
    if j == 0:
        return 0.0
    for _ in range(j - 1):
        t0, t1, d0, d1 = t1, 2.0 * x * t1 - t0, d1, 2.0 * t1 + 2.0 * x * d1 - d0
    return d1


def coefficients(s: int, eps: float):
    """(w0, w1, mu, nu, mut) with mu[j], nu[j], mut[j] for stages j = 1..s
    (index 0 unused; stage 1 has mu = 1, nu = 0)."""
    w0 = 1.0 + eps / (s * s)
    w1 = cheb(s, w0) / dcheb(s, w0)
    b = [1.0 / cheb(j, w0) for j in range(s + 1)]
    mu = np.zeros(s + 1)
    nu = np.zeros(s + 1)
    mut = np.zeros(s + 1)
    mu[1], nu[1], mut[1] = 1.0, 0.0, w1 / w0
    for j in range(2, s + 1):
        mu[j] = 2.0 * w0 * b[j] / b[j - 1]
        nu[j] = -b[j] / b[j - 2]
        mut[j] = 2.0 * w1 * b[j] / b[j - 1]
    return w0, w1, mu, nu, mut


def beta(s: int, eps: float) -> float:
    """Length of the real stability interval [-beta, 0]."""
    w0, w1, *_ = coefficients(s, eps)
    return (1.0 + w0) / w1


def coefficients2(s: int, eps: float):
    """Second-order damped Chebyshev recurrence (RKC2): with w0 = 1 + eps/s^2,
    w1 = T_s'(w0)/T_s''(w0), b_j = T_j''(w0)/T_j'(w0)^2 (b_0 = b_1 = b_2),
    a_j = 1 - b_j T_j(w0):
      Y_1 = Y_0 + mut_1 tau K F(Y_0),  mut_1 = b_1 w1,
      Y_j = (1 - mu_j - nu_j) Y_0 + mu_j Y_{j-1} + nu_j Y_{j-2}
            + mut_j tau K F(Y_{j-1}) + gam_j tau K F(Y_0),
      mu_j = 2 b_j w0 / b_{j-1}, nu_j = -b_j / b_{j-2}, mut_j = 2 b_j w1 / b_{j-1},
      gam_j = -a_{j-1} mut_j,
    so that a linear mode is multiplied by P_s(z) = a_s + b_s T_s(w0 + w1 z),
    with P_s(0) = 1, P_s'(0) = 1, P_s''(0) = 1.  Returns (w0, w1, mu, nu, mut, gam)
    indexed by stage j = 1..s."""
    w0 = 1.0 + eps / (s * s)
    T = [cheb(j, w0) for j in range(s + 1)]
    d1 = [dcheb(j, w0) for j in range(s + 1)]
    d2 = [ddcheb(j, w0) for j in range(s + 1)]
    w1 = d1[s] / d2[s]
    b = [0.0] * (s + 1)
    for j in range(2, s + 1):
        b[j] = d2[j] / (d1[j] * d1[j])
    b[0] = b[1] = b[2]
    a = [1.0 - b[j] * T[j] for j in range(s + 1)]
    mu = np.zeros(s + 1)
    nu = np.zeros(s + 1)
    mut = np.zeros(s + 1)
    gam = np.zeros(s + 1)
    mu[1], mut[1] = 1.0, b[1] * w1
    for j in range(2, s + 1):
        mu[j] = 2.0 * b[j] * w0 / b[j - 1]
        nu[j] = -b[j] / b[j - 2]
        mut[j] = 2.0 * b[j] * w1 / b[j - 1]
        gam[j] = -a[j - 1] * mut[j]
    return w0, w1, mu, nu, mut, gam, a, b


def beta2(s: int, eps: float) -> float:
    w0, w1, *_ = coefficients2(s, eps)
    return (1.0 + w0) / w1


def ddcheb(j: int, x: float) -> float:
    """T_j''(x) by differentiating the recurrence twice."""
    t0, t1 = 1.0, x
    d0, d1 = 0.0, 1.0
    e0, e1 = 0.0, 0.0
    if j < 2:
        return 0.0
    for _ in range(j - 1):
        t2 = 2.0 * x * t1 - t0
        d2 = 2.0 * t1 + 2.0 * x * d1 - d0
        e2 = 4.0 * d1 + 2.0 * x * e1 - e0
        t0, t1, d0, d1, e0, e1 = t1, t2, d1, d2, e1, e2
    return e1


def window2(rowptr, col, theta, K: float, tau: float, s: int, eps: float):
    """Y_s of the second-order recurrence for the flux part; returns (Y_s, F(Y_0))."""
    _, _, mu, nu, mut, gam, _, _ = coefficients2(s, eps)
    y0 = np.asarray(theta, dtype=np.float64).copy()
    F0 = flux_sum(rowptr, col, y0)
    y_prev2 = y0
    y_prev = y0 + mut[1] * tau * K * F0
    for j in range(2, s + 1):
        F = flux_sum(rowptr, col, y_prev)
        kap = 1.0 - mu[j] - nu[j]
        # mu Y_{j-1} + nu Y_{j-2} + kap Y_0 with mu + nu + kap = 1, as increments
        y = y_prev + nu[j] * (y_prev2 - y_prev) + kap * (y0 - y_prev) + tau * K * (mut[j] * F + gam[j] * F0)
        y_prev2, y_prev = y_prev, y
    return y_prev, F0


def window(rowptr, col, theta, K: float, tau: float, s: int, eps: float, coeffs=None):
    """Y_s for the flux part over one window; returns (Y_s, F(Y_0))."""
    mu, nu, mut = (coeffs if coeffs is not None else coefficients(s, eps)[2:])
    y0 = np.asarray(theta, dtype=np.float64).copy()
    F0 = flux_sum(rowptr, col, y0)
    y_prev2 = y0
    y_prev = y0 + mut[1] * tau * K * F0
    for j in range(2, s + 1):
        F = flux_sum(rowptr, col, y_prev)
        # mu_j Y_{j-1} + nu_j Y_{j-2} with mu_j = 1 - nu_j, as an increment
        y = y_prev + nu[j] * (y_prev2 - y_prev) + mut[j] * tau * K * F
        y_prev2, y_prev = y_prev, y
    return y_prev, F0
