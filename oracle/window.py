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
conservation and the uniform fixed point.  The general stage form with free
coefficients (window_general, its adjoint gradient window_grad and
stability_polynomial, used to train windows) is pinned by reproducing both
recurrences and their closed-form stability polynomials, and by central
differences of the loss and of the flux sum (flux_vjp); the adjoint through a
chain of windows (rollout_grad) by central differences of rollout_loss.
"""
from __future__ import annotations

import math

import numpy as np

from . import flux_sum, flux_vjp


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


# ---- windows with arbitrary stage coefficients (trained windows) ----------------
#
# The general stage of both recurrences above, written on the window's change
# z_j = Y_j - Y_0 (z_0 = 0), with a_j = mut_j tau K and g_j = gam_j tau K:
#   z_1 = a_1 F(Y_0),
#   z_j = z_{j-1} + nu_j (z_{j-2} - z_{j-1}) - kap_j z_{j-1} + a_j F(Y_{j-1}) + g_j F(Y_0),
# which is Y_j = (1 - mu_j - nu_j) Y_0 + mu_j Y_{j-1} + nu_j Y_{j-2} + ... with
# kap_j = 1 - mu_j - nu_j.  Training treats nu, mut, kap, gam (stages 1..s) as
# free parameters.


def window_general(rowptr, col, theta, K: float, tau: float, coeffs):
    """Stages of one window with coefficients (nu, mut, kap, gam), each indexed
    j = 0..s (index 0 unused).  Returns (z, F): z[j] = Y_j - Y_0 for j = 0..s and
    F[j] = F(Y_{j-1}) for j = 1..s (F[1] = F(Y_0))."""
    nu, mut, kap, gam = (np.asarray(c, dtype=np.float64) for c in coeffs)
    s = len(nu) - 1
    y0 = np.asarray(theta, dtype=np.float64)
    z = [np.zeros_like(y0)]
    F = [None, flux_sum(rowptr, col, y0)]
    z.append(mut[1] * tau * K * F[1])
    for j in range(2, s + 1):
        F.append(flux_sum(rowptr, col, y0 + z[j - 1]))
        z.append(z[j - 1] + nu[j] * (z[j - 2] - z[j - 1]) - kap[j] * z[j - 1]
                 + tau * K * (mut[j] * F[j] + gam[j] * F[1]))
    return z, F


def window_loss(T0, T1, z_s, Tmax: float, power: int = 2) -> float:
    """Training loss of a window: the mean of the relative error of the end
    temperatures to the given even power, mean_i ((T0_i + Tmax z_s,i - T1_i) / T0_i)^p."""
    r = (np.asarray(T0) + Tmax * z_s - np.asarray(T1)) / np.asarray(T0)
    return float(np.mean(r ** power))


def window_grad(rowptr, col, T0, T1, Tmax: float, K: float, tau: float, coeffs, power: int = 2):
    """Loss (window_loss, exponent `power`) of the window started from T0 against the target T1,
    and its gradient with respect to (nu, mut, kap, gam), by the adjoint of the
    stage recurrence: with lam_j = dL/dz_j, going down from j = s,
      dL/dnu_j = <lam_j, z_{j-2} - z_{j-1}>,  dL/dkap_j = -<lam_j, z_{j-1}>,
      dL/dmut_j = tau K <lam_j, F(Y_{j-1})>,  dL/dgam_j = tau K <lam_j, F(Y_0)>,
      lam_{j-1} += (1 - nu_j - kap_j) lam_j + a_j J(Y_{j-1})^T lam_j,
      lam_{j-2} += nu_j lam_j,
    J the Jacobian of the flux sum (flux_vjp); Y_0 is data, not a parameter.
    Returns (loss, [g_nu, g_mut, g_kap, g_gam]) with entries for j = 0..s
    (0 for j = 0, and for nu_1, kap_1, gam_1, which stage 1 does not use)."""
    nu, mut, kap, gam = (np.asarray(c, dtype=np.float64) for c in coeffs)
    s = len(nu) - 1
    T0 = np.asarray(T0, dtype=np.float64)
    T1 = np.asarray(T1, dtype=np.float64)
    y0 = T0 / Tmax
    z, F = window_general(rowptr, col, y0, K, tau, coeffs)
    n = T0.shape[0]
    loss = window_loss(T0, T1, z[s], Tmax, power)
    lam = [np.zeros(n) for _ in range(s + 1)]
    # d/dz_s of mean(r^p), r = (T0 + Tmax z_s - T1) / T0
    r = (T0 + Tmax * z[s] - T1) / T0
    lam[s] = power * r ** (power - 1) * Tmax / T0 / n
    g = [np.zeros(s + 1) for _ in range(4)]
    for j in range(s, 1, -1):
        lj = lam[j]
        g[0][j] = lj @ (z[j - 2] - z[j - 1])
        g[1][j] = tau * K * (lj @ F[j])
        g[2][j] = -(lj @ z[j - 1])
        g[3][j] = tau * K * (lj @ F[1])
        lam[j - 1] += (1.0 - nu[j] - kap[j]) * lj + mut[j] * tau * K * flux_vjp(rowptr, col, y0 + z[j - 1], lj)
        lam[j - 2] += nu[j] * lj
    g[1][1] = tau * K * (lam[1] @ F[1])
    return loss, g


def stability_polynomial(coeffs, x):
    """P(x) of the stages on the linear test mode tau K F(Y) = -x Y (Y_0 = 1):
    the factor one window applies to a mode of rate lambda, x = tau lambda."""
    nu, mut, kap, gam = (np.asarray(c, dtype=np.float64) for c in coeffs)
    s = len(nu) - 1
    x = np.asarray(x, dtype=np.float64)
    zm2 = np.zeros_like(x)
    zm1 = -mut[1] * x
    for j in range(2, s + 1):
        z = zm1 + nu[j] * (zm2 - zm1) - kap[j] * zm1 - mut[j] * x * (1.0 + zm1) - gam[j] * x
        zm2, zm1 = zm1, z
    return 1.0 + zm1


def coefficient_sets(s: int, order: int, eps: float):
    """(nu, mut, kap, gam) of the damped Chebyshev recurrence of the given order
    in the general stage form (kap = gam = 0 for order 1)."""
    if order == 1:
        _, _, mu, nu, mut = coefficients(s, eps)
        return [nu.copy(), mut.copy(), np.zeros(s + 1), np.zeros(s + 1)]
    _, _, mu, nu, mut, gam, _, _ = coefficients2(s, eps)
    kap = 1.0 - mu - nu
    kap[0] = kap[1] = 0.0
    return [nu.copy(), mut.copy(), kap, gam.copy()]


# ---- rollouts: chains of windows (training against a trajectory) -------------
#
# K windows in a row, each started from the previous one's end: theta_0 =
# T_in / Tmax, theta_w = theta_{w-1} + z_s(theta_{w-1}).  Loss against the plain
# method's trajectory T*_1..T*_K:
#   L = sum_w mean_i ((Tmax theta_w,i - T*_w,i) / T*_w,i)^p.
# Its adjoint runs the windows backwards: with Lam_w = dL/dtheta_w, window w's
# stage adjoint starts from lam_s = Lam_w and, besides the coefficient
# gradients, gives dL/dtheta_{w-1} through the window:
#   Lam_w + sum_{j>=1} a_j J(Y_{j-1})^T lam_j + J(Y_0)^T sum_{j>=2} g_j lam_j,
# (Y_{j-1} = Y_0 + z_{j-1} depends on Y_0 directly), to which the loss term of
# window w-1 is added.


def rollout_loss(rowptr, col, T_in, T_targets, Tmax: float, K: float, tau: float, coeffs, power: int = 2):
    """Loss of len(T_targets) chained windows started from T_in."""
    th = np.asarray(T_in, dtype=np.float64) / Tmax
    s = len(coeffs[0]) - 1
    L = 0.0
    for Tt in T_targets:
        z, _ = window_general(rowptr, col, th, K, tau, coeffs)
        th = th + z[s]
        r = (Tmax * th - Tt) / Tt
        L += float(np.mean(r ** power))
    return L


def rollout_grad(rowptr, col, T_in, T_targets, Tmax: float, K: float, tau: float, coeffs, power: int = 2):
    """rollout_loss and its gradient with respect to (nu, mut, kap, gam), by the
    adjoint through the chain of windows (see above)."""
    nu, mut, kap, gam = (np.asarray(c, dtype=np.float64) for c in coeffs)
    s = len(nu) - 1
    n = np.asarray(T_in).shape[0]
    ths = [np.asarray(T_in, dtype=np.float64) / Tmax]
    stages = []
    L = 0.0
    for Tt in T_targets:
        z, F = window_general(rowptr, col, ths[-1], K, tau, coeffs)
        stages.append((z, F))
        ths.append(ths[-1] + z[s])
        r = (Tmax * ths[-1] - Tt) / Tt
        L += float(np.mean(r ** power))
    g = [np.zeros(s + 1) for _ in range(4)]
    aK, gK = tau * K * mut, tau * K * gam
    Lam = np.zeros(n)
    for w in range(len(T_targets) - 1, -1, -1):
        Tt = np.asarray(T_targets[w], dtype=np.float64)
        r = (Tmax * ths[w + 1] - Tt) / Tt
        Lam = Lam + power * r ** (power - 1) * Tmax / Tt / n
        y0 = ths[w]
        z, F = stages[w]
        lam = [np.zeros(n) for _ in range(s + 1)]
        lam[s] = Lam.copy()
        mu = np.zeros(n)       # sum_j a_j J(Y_{j-1})^T lam_j for j >= 2
        gsum = np.zeros(n)     # sum_{j>=2} g_j lam_j
        for j in range(s, 1, -1):
            lj = lam[j]
            g[0][j] += lj @ (z[j - 2] - z[j - 1])
            g[1][j] += tau * K * (lj @ F[j])
            g[2][j] += -(lj @ z[j - 1])
            g[3][j] += tau * K * (lj @ F[1])
            v = aK[j] * flux_vjp(rowptr, col, y0 + z[j - 1], lj)
            lam[j - 1] += (1.0 - nu[j] - kap[j]) * lj + v
            lam[j - 2] += nu[j] * lj
            mu += v
            gsum += gK[j] * lj
        g[1][1] += tau * K * (lam[1] @ F[1])
        mu += flux_vjp(rowptr, col, y0, aK[1] * lam[1] + gsum)
        Lam = Lam + mu
    return L, g
