"""Pins of the FP64 Chebyshev window reference (oracle/window.py) against
closed forms: the Chebyshev polynomials cos(s arccos x) / cosh(s arccosh x),
the stability polynomial of the recurrence on a linear lattice mode, the sum
of temperatures (Eq. HeatTransport conserves it) and the uniform fixed point."""
import math

import numpy as np
import pytest

import oracle
from oracle import window as W
from paper_1810_12357_gb300 import inputs as I


def T_closed(s, x):
    if abs(x) <= 1.0:
        return math.cos(s * math.acos(x))
    if x > 1.0:
        return math.cosh(s * math.acosh(x))
    return (-1.0) ** s * math.cosh(s * math.acosh(-x))


def P_closed(s, eps, z):
    w0 = 1.0 + eps / (s * s)
    # w1 = T_s(w0) / T_s'(w0) with T_s'(x) = s sinh(s arccosh x) / sinh(arccosh x) for x > 1
    a = math.acosh(w0)
    w1 = math.cosh(s * a) * math.sinh(a) / (s * math.sinh(s * a))
    return T_closed(s, w0 + w1 * z) / T_closed(s, w0)


@pytest.mark.parametrize("s", [2, 3, 4, 6])
def test_recurrence_matches_closed_form(s):
    for x in (-0.9, -0.3, 0.2, 0.95, 1.0, 1.02, 1.3):
        assert W.cheb(s, x) == pytest.approx(T_closed(s, x), rel=1e-12, abs=1e-12)
    w0, w1, mu, nu, mut = W.coefficients(s, 0.05)
    a = math.acosh(w0)
    assert w1 == pytest.approx(math.cosh(s * a) * math.sinh(a) / (s * math.sinh(s * a)), rel=1e-12)
    for j in range(2, s + 1):
        assert mu[j] + nu[j] == pytest.approx(1.0, abs=1e-14)   # affine: the sum of theta is kept


@pytest.mark.parametrize("s", [3, 4, 5])
def test_stability_polynomial(s):
    eps = 0.05
    # first order: P(0) = 1, P'(0) = 1
    h = 1e-5
    assert P_closed(s, eps, 0.0) == pytest.approx(1.0, abs=1e-14)
    assert (P_closed(s, eps, h) - P_closed(s, eps, -h)) / (2 * h) == pytest.approx(1.0, rel=1e-8)
    b = W.beta(s, eps)
    assert b == pytest.approx((2.0 - 4.0 * eps / 3.0) * s * s, rel=0.02)
    zs = np.linspace(-b, 0.0, 2001)
    assert max(abs(P_closed(s, eps, z)) for z in zs) <= 1.0 + 1e-12
    assert abs(P_closed(s, eps, -1.05 * b)) > 1.0


def _fcc(nc):
    a = I.CU_A
    x = I.fcc_lattice(nc, nc, nc, a)
    box = np.array([nc * a] * 3)
    per = np.array([1, 1, 1], dtype=np.int32)
    rowptr, col = oracle.neighbors(x, box, per, 4.0)
    return a, x, rowptr, col


def test_linear_mode_follows_the_stability_polynomial():
    # a small sin(k x) mode on the perfect lattice decays over one window by
    # exactly P_s(-tau lambda_k), lambda_k = K c(theta) sum_j (1 - cos k.r_j)
    a, x, rowptr, col = _fcc(6)
    shell = I.fcc_shell_vectors(a, 4.0)
    th0, amp, K = 0.003, 1e-9, 1.0
    c = 1.0 - 2.0 * th0 * (1.0 - th0)
    s, eps = 4, 0.05
    for kc in (6, 3, 2):                      # k = 2 pi / (kc a): long to short waves
        k = 2.0 * math.pi / (kc * a)
        lam = K * c * float((1.0 - np.cos(k * shell[:, 0])).sum())
        mode = np.sin(k * x[:, 0])
        for tau in (0.02, 0.5, 0.9 * W.beta(s, eps) / lam):
            y, _ = W.window(rowptr, col, th0 + amp * mode, K, tau, s, eps)
            a1 = float((y - th0) @ mode / (mode @ mode))
            assert a1 == pytest.approx(amp * P_closed(s, eps, -tau * lam), rel=2e-5, abs=1e-17)


def test_conservation_and_fixed_point():
    s = I.hot_spot_system(5, 3, peak=9000.0)
    rowptr, col = oracle.neighbors(s.x, s.box, s.periodic, 4.0)
    th = s.Te / 2.0e4
    y, F0 = W.window(rowptr, col, th, 20.0, 0.02, 4, 0.05)
    assert abs(y.sum() - th.sum()) < 1e-13 * th.sum()
    assert abs(F0.sum()) < 1e-12
    assert y.max() < th.max()
    u = np.full(s.n, 0.0617)
    yu, _ = W.window(rowptr, col, u, 20.0, 0.02, 4, 0.05)
    assert np.all(yu == u)


def test_l_point_mode_bounded_inside_the_interval():
    # the most unstable lattice mode (rate 24 K c) stays bounded while
    # tau lambda_L <= beta and grows beyond it
    a, x, rowptr, col = _fcc(4)
    mode = np.cos(np.pi * x.sum(axis=1) / a)
    th0, amp, K = 0.003, 1e-9, 1.0
    lam = 24.0 * K * (1.0 - 2.0 * th0 * (1.0 - th0))
    s, eps = 4, 0.05
    b = W.beta(s, eps)
    for r, bounded in ((0.98, True), (1.10, False)):
        y = th0 + amp * mode
        for _ in range(20):
            y, _ = W.window(rowptr, col, y, K, r * b / lam, s, eps)
        a1 = float((y - th0) @ mode / (mode @ mode))
        assert (abs(a1) <= amp) == bounded


def test_window_against_plain_substeps_on_the_track():
    # how far one Chebyshev window (4 stages, 16 substeps of the bench's dt) is
    # from the 16 explicit substeps it replaces, along the plain trajectory of
    # the track profile: several per cent in the first window (the heat front
    # moves by ~70 % of the local temperature within one window, where the two
    # first-order maps differ in their error constants), well under 1 % once the
    # profile has spread
    s = I.track_system(24, 2, r0=20.0)
    p = I.params_track()
    sim = oracle.OracleSim(p, s.box, s.periodic, s.mass_amu, s.type)
    sim.set_te(s.Te)
    sim.build(s.x, s.v)
    K, Tmax, dt = sim.K, p["Tmax"], p["dt_sub"]
    T = s.Te.copy()
    errs = []
    for w in range(20):
        y, _ = W.window(sim.rowptr, sim.col, T / Tmax, K, 16 * dt, 4, 0.05)
        Tn = T.copy()
        zeros = np.zeros(s.n)
        oracle.substeps(sim.rowptr, sim.col, Tn, zeros, np.zeros(s.n, np.uint8), zeros.copy(), 16, dt, Tmax, K,
                        0.0, 0.0)
        errs.append(float(np.max(np.abs(y * Tmax - Tn) / Tn)))
        T = Tn
    assert errs[0] > 0.05
    assert errs[19] < 1e-3
    assert all(errs[k + 1] < errs[k] for k in range(0, 19, 3))


def P2_closed(s, eps, z):
    # P_s(z) = a_s + b_s T_s(w0 + w1 z), w1 = T_s'(w0)/T_s''(w0), b_s = T_s''/T_s'^2,
    # a_s = 1 - b_s T_s(w0); T_s', T_s'' from x = cosh(t): T_s = cosh(s t),
    # T_s' = s sinh(s t)/sinh t, T_s'' = (s^2 cosh(s t) sinh t - s sinh(s t) cosh t) / sinh^3 t
    w0 = 1.0 + eps / (s * s)
    t = math.acosh(w0)
    Ts = math.cosh(s * t)
    d1 = s * math.sinh(s * t) / math.sinh(t)
    d2 = (s * s * math.cosh(s * t) * math.sinh(t) - s * math.sinh(s * t) * math.cosh(t)) / math.sinh(t) ** 3
    w1 = d1 / d2
    b = d2 / (d1 * d1)
    return (1.0 - b * Ts) + b * T_closed(s, w0 + w1 * z)


@pytest.mark.parametrize("s", [4, 7, 10])
def test_second_order_stability_polynomial(s):
    eps = 2.0 / 13.0
    h = 1e-4
    assert P2_closed(s, eps, 0.0) == pytest.approx(1.0, abs=1e-13)
    assert (P2_closed(s, eps, h) - P2_closed(s, eps, -h)) / (2 * h) == pytest.approx(1.0, rel=1e-7)
    d2 = (P2_closed(s, eps, h) - 2 * P2_closed(s, eps, 0.0) + P2_closed(s, eps, -h)) / (h * h)
    assert d2 == pytest.approx(1.0, rel=1e-4)
    b = W.beta2(s, eps)
    assert b == pytest.approx(0.653 * s * s, rel=0.08)
    zs = np.linspace(-b, 0.0, 2001)
    assert max(abs(P2_closed(s, eps, z)) for z in zs) <= 1.0 + 1e-12
    # the recurrence's coefficients reproduce the same polynomial on a scalar mode
    _, _, mu, nu, mut, gam, _, _ = W.coefficients2(s, eps)
    for z in (-0.3 * b, -0.8 * b):
        y0, F0 = 1.0, z
        ym2, ym1 = y0, y0 + mut[1] * F0
        for j in range(2, s + 1):
            y = (1 - mu[j] - nu[j]) * y0 + mu[j] * ym1 + nu[j] * ym2 + mut[j] * z * ym1 + gam[j] * z * y0
            ym2, ym1 = ym1, y
        assert ym1 == pytest.approx(P2_closed(s, eps, z), rel=1e-10, abs=1e-12)


def test_second_order_window_on_a_lattice_mode_and_invariants():
    a, x, rowptr, col = _fcc(6)
    shell = I.fcc_shell_vectors(a, 4.0)
    th0, amp, K = 0.003, 1e-9, 1.0
    c = 1.0 - 2.0 * th0 * (1.0 - th0)
    s, eps = 7, 2.0 / 13.0
    k = 2.0 * math.pi / (3 * a)
    lam = K * c * float((1.0 - np.cos(k * shell[:, 0])).sum())
    mode = np.sin(k * x[:, 0])
    for tau in (0.05, 0.9 * W.beta2(s, eps) / lam):
        y, _ = W.window2(rowptr, col, th0 + amp * mode, K, tau, s, eps)
        a1 = float((y - th0) @ mode / (mode @ mode))
        assert a1 == pytest.approx(amp * P2_closed(s, eps, -tau * lam), rel=2e-5, abs=1e-17)
    hs = I.hot_spot_system(5, 3, peak=9000.0)
    rp, cl = oracle.neighbors(hs.x, hs.box, hs.periodic, 4.0)
    th = hs.Te / 2.0e4
    y, _ = W.window2(rp, cl, th, 20.0, 0.02, s, eps)
    assert abs(y.sum() - th.sum()) < 1e-13 * th.sum()
    u = np.full(hs.n, 0.0617)
    yu, _ = W.window2(rp, cl, u, 20.0, 0.02, s, eps)
    assert np.all(yu == u)


# ---- windows with free stage coefficients (the trained window) ----------------

def _small_system(seed=3):
    # 5^3 FCC cells (500 atoms) with a smooth profile and a random ripple,
    # theta within (0.01, 0.5)
    _, x, rowptr, col = _fcc(5)
    rng = np.random.default_rng(seed)
    box = 5 * 3.615
    th = 0.05 + 0.3 * np.exp(-np.sum((x - 0.5 * box) ** 2, axis=1) / 30.0) + 0.02 * rng.random(x.shape[0])
    return rowptr, col, th


def test_pair_derivative_matches_differences():
    for a, b in [(0.1, 0.3), (0.5, 0.02), (0.7, 0.7), (0.01, 0.9), (0.33, 0.31)]:
        h = 1e-6
        fd = (oracle.pair_flux(a + h, b) - oracle.pair_flux(a - h, b)) / (2 * h)
        assert oracle.pair_dflux_a(a, b) == pytest.approx(fd, rel=1e-8, abs=1e-10)
    # at a = b the slope is -(a^2 + (1 - a)^2), the linearisation of the pair term
    assert oracle.pair_dflux_a(0.2, 0.2) == pytest.approx(-(0.04 + 0.64), rel=1e-15)


def test_flux_vjp_is_the_transposed_jacobian():
    rowptr, col, th = _small_system()
    rng = np.random.default_rng(1)
    u, v = rng.normal(size=th.size), rng.normal(size=th.size)
    h = 1e-6
    Jv = (oracle.flux_sum(rowptr, col, th + h * v) - oracle.flux_sum(rowptr, col, th - h * v)) / (2 * h)
    assert np.dot(u, Jv) == pytest.approx(np.dot(oracle.flux_vjp(rowptr, col, th, u), v), rel=1e-7)
    # sum_i F_i = 0 for every state, so J^T 1 = 0
    assert np.max(np.abs(oracle.flux_vjp(rowptr, col, th, np.ones(th.size)))) < 1e-12


@pytest.mark.parametrize("order", [1, 2])
def test_general_stages_reproduce_both_recurrences(order):
    rowptr, col, th = _small_system()
    K, tau, s = 40.0, 0.05, 6
    C = W.coefficient_sets(s, order, 0.05 if order == 1 else 2 / 13)
    z, _ = W.window_general(rowptr, col, th, K, tau, C)
    if order == 1:
        y, _ = W.window(rowptr, col, th, K, tau, s, 0.05)
    else:
        y, _ = W.window2(rowptr, col, th, K, tau, s, 2 / 13)
    # same arithmetic in another rounding order (-kap z against kap (Y_0 - Y))
    assert np.max(np.abs(th + z[s] - y)) < 1e-10
    # and the general stability polynomial is the closed form of each family
    for x in (0.0, 0.7, 3.0, 11.0, 0.5 * (W.beta(s, 0.05) if order == 1 else W.beta2(s, 2 / 13))):
        want = P_closed(s, 0.05, -x) if order == 1 else P2_closed(s, 2 / 13, -x)
        assert W.stability_polynomial(C, x) == pytest.approx(want, rel=1e-11, abs=1e-13)


@pytest.mark.parametrize("power", [2, 4])
def test_window_gradient_matches_differences(power):
    rowptr, col, th = _small_system()
    K, tau, s, Tmax = 40.0, 0.06, 5, 20000.0
    T0 = th * Tmax
    C = W.coefficient_sets(s, 2, 2 / 13)
    # target: the same window with perturbed coefficients, so the loss is not at a minimum
    Ct = [c * (1.0 + 0.05 * np.sin(np.arange(c.size) + k)) for k, c in enumerate(C)]
    zt, _ = W.window_general(rowptr, col, th, K, tau, Ct)
    T1 = T0 + Tmax * zt[s]
    loss, g = W.window_grad(rowptr, col, T0, T1, Tmax, K, tau, C, power)
    assert loss > 0
    checked = 0
    for k in range(4):
        for j in range(1, s + 1):
            if j == 1 and k != 1:
                assert g[k][j] == 0.0   # stage 1 uses mut_1 only
                continue
            h = 1e-6 * max(abs(C[k][j]), 1e-3)
            Cp = [c.copy() for c in C]
            Cm = [c.copy() for c in C]
            Cp[k][j] += h
            Cm[k][j] -= h
            lp = W.window_loss(T0, T1, W.window_general(rowptr, col, th, K, tau, Cp)[0][s], Tmax, power)
            lm = W.window_loss(T0, T1, W.window_general(rowptr, col, th, K, tau, Cm)[0][s], Tmax, power)
            fd = (lp - lm) / (2 * h)
            assert g[k][j] == pytest.approx(fd, rel=2e-5, abs=1e-9 * abs(loss) / h), (k, j)
            checked += 1
    assert checked == 4 * s - 3


@pytest.mark.parametrize("power", [2, 4])
def test_rollout_gradient_matches_differences(power):
    # three chained windows against a trajectory the window itself would not
    # reproduce (other coefficients): the adjoint through the chain against
    # central differences of the rollout loss, for every coefficient
    rowptr, col, th = _small_system(5)
    # tau K lambda_max about 11.5, inside the 5-stage second-order interval (16):
    # the chained windows stay bounded
    K, tau, s, Tmax = 40.0, 0.02, 5, 20000.0
    C = W.coefficient_sets(s, 2, 2 / 13)
    Ct = [c * (1.0 + 0.05 * np.cos(np.arange(c.size) + 2 * k)) for k, c in enumerate(C)]
    T_in = th * Tmax
    targets, y = [], th.copy()
    for _ in range(3):
        z, _ = W.window_general(rowptr, col, y, K, tau, Ct)
        y = y + z[s]
        targets.append(Tmax * y)
    loss, g = W.rollout_grad(rowptr, col, T_in, targets, Tmax, K, tau, C, power)
    assert loss == pytest.approx(W.rollout_loss(rowptr, col, T_in, targets, Tmax, K, tau, C, power), rel=1e-14)
    for k in range(4):
        for j in range(1, s + 1):
            if j == 1 and k != 1:
                assert g[k][j] == 0.0
                continue
            h = 1e-6 * max(abs(C[k][j]), 1e-3)
            Cp = [c.copy() for c in C]
            Cm = [c.copy() for c in C]
            Cp[k][j] += h
            Cm[k][j] -= h
            fd = (W.rollout_loss(rowptr, col, T_in, targets, Tmax, K, tau, Cp, power)
                  - W.rollout_loss(rowptr, col, T_in, targets, Tmax, K, tau, Cm, power)) / (2 * h)
            assert g[k][j] == pytest.approx(fd, rel=2e-5, abs=1e-9 * abs(loss) / h), (k, j)
