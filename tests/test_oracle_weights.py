"""Pins of the oracle's distance-weighted pair rates (ehc_params.rate_shell_n,
an optional variant: the paper's K_ij is one rate for all pairs).  w_ij =
S2 / (n_shell r_ij^2): on the 18-neighbour FCC shell at r_c = 4 A (S2 = 12 a^2)
the nearest neighbours get 4/3 and the second shell 2/3; the weights are
symmetric; pair fluxes stay odd, so sum_i T_i is kept; a sin mode decays at
the weighted lattice sum c K sum_j w_j (1 - cos k r_j), and in the long-wave
limit at the same rate as with uniform rates."""
import math

import numpy as np
import pytest

import oracle
from paper_1810_12357_gb300 import inputs as I


def _lattice(nx=6, ny=3, nz=3, disp=0.0, seed=0):
    a = I.CU_A
    x = I.fcc_lattice(nx, ny, nz, a)
    box = np.array([nx * a, ny * a, nz * a])
    if disp > 0:
        x = I.wrap(x + np.random.default_rng(seed).normal(0, disp, x.shape), box, np.array([1, 1, 1]))
    per = np.array([1, 1, 1], dtype=np.int32)
    rowptr, col = oracle.neighbors(x, box, per, 4.0)
    return a, x, box, per, rowptr, col


def test_fcc_shell_weights_and_second_moment():
    a, x, box, per, rowptr, col = _lattice()
    S2 = I.fcc_shell_s2(a, 4.0)
    assert S2 == pytest.approx(12 * a * a, rel=1e-12)
    w = oracle.pair_weights(x, box, per, rowptr, col, S2, 18)
    q, Lq = oracle.quantize(x, box, per)
    i = np.repeat(np.arange(x.shape[0]), np.diff(rowptr))
    d = (q[col] - q[i]).astype(np.float64)
    d -= np.round(d / Lq) * Lq
    r2 = (d * d).sum(1) / 2.0 ** 40
    near = r2 < 0.75 * a * a
    assert near.sum() == 12 * x.shape[0] and (~near).sum() == 6 * x.shape[0]
    # the grid rounds each coordinate by <= 2^-21 A, so r^2 is off by at most
    # 2 sqrt(3) 2^-20 / r_1 = 1.3e-6 relative: weights within 2.5e-6 of the ideal
    assert np.max(np.abs(w[near] - 4.0 / 3.0)) < 2.5e-6
    assert np.max(np.abs(w[~near] - 2.0 / 3.0)) < 2.5e-6
    # each atom's weighted second moment is the shell's S2 (r^2 w is exactly S2/18 per pair)
    m2 = np.bincount(i, weights=w * r2)
    assert np.max(np.abs(m2 - S2)) < 1e-12 * S2


def test_weights_are_symmetric_and_conserve():
    a, x, box, per, rowptr, col = _lattice(disp=0.08, seed=3)
    w = oracle.pair_weights(x, box, per, rowptr, col, I.fcc_shell_s2(a, 4.0), 18)
    n = x.shape[0]
    i = np.repeat(np.arange(n), np.diff(rowptr))
    key = {(int(a_), int(b_)): float(v) for a_, b_, v in zip(i, col, w)}
    assert all(key[(b_, a_)] == v for (a_, b_), v in key.items())
    rng = np.random.default_rng(1)
    T = 300.0 + 2000.0 * rng.random(n)
    T0 = T.copy()
    zeros = np.zeros(n)
    st, _ = oracle.substeps(rowptr, col, T, zeros, np.zeros(n, np.uint8), zeros.copy(), 200, 1e-3, 1e5, 40.0,
                            0.0, 0.0, weights=w)
    assert st == 200
    assert abs(T.sum() - T0.sum()) < 1e-12 * T0.sum()
    assert np.max(np.abs(T - T0)) > 1.0


def _decay(ncx, k_cells, n_sub, weights, T0=300.0, Tmax=2.0e4):
    a = I.CU_A
    x = I.fcc_lattice(ncx, 3, 3, a)
    box = np.array([ncx * a, 3 * a, 3 * a])
    per = np.array([1, 1, 1], dtype=np.int32)
    rowptr, col = oracle.neighbors(x, box, per, 4.0)
    S2 = I.fcc_shell_s2(a, 4.0)
    w = oracle.pair_weights(x, box, per, rowptr, col, S2, 18) if weights else None
    k = 2 * math.pi / (k_cells * a)
    basis = np.sin(k * x[:, 0])
    T = T0 + basis
    n = x.shape[0]
    K, dt = 40.0, 1e-3
    zeros = np.zeros(n)
    a0 = float((T - T0) @ basis / (basis @ basis))
    oracle.substeps(rowptr, col, T, zeros, np.zeros(n, np.uint8), zeros.copy(), n_sub, dt, Tmax, K, 0.0, 0.0,
                    weights=w)
    a1 = float((T - T0) @ basis / (basis @ basis))
    th = T0 / Tmax
    c = 1 - 2 * th * (1 - th)
    shell = I.fcc_shell_vectors(a, 4.0)
    r = np.sqrt((shell * shell).sum(1))
    ws = S2 / (18 * r * r) if weights else np.ones(len(r))
    lam = c * K * float((ws * (1 - np.cos(k * shell[:, 0]))).sum())
    return a0, a1, lam, dt, k, c, K, S2


def test_weighted_sin_mode_follows_the_lattice_sum():
    a0, a1, lam, dt, *_ = _decay(10, 10, 400, True)
    assert a1 == pytest.approx(a0 * (1 - dt * lam) ** 400, rel=1e-6)
    # and the weighted rate differs from the uniform one at this wavelength
    _, _, lam_u, *_ = _decay(10, 10, 1, False)
    assert abs(lam / lam_u - 1.0) > 1e-3


def test_long_wave_rate_is_that_of_uniform_rates():
    # sum_j w_j (k.r_j)^2 = k^2 S2 / 3 for both weightings: the same conductivity
    _, _, lam_w, dt, k, c, K, S2 = _decay(40, 40, 1, True)
    _, _, lam_u, *_ = _decay(40, 40, 1, False)
    assert lam_w == pytest.approx(c * K * k * k * S2 / 6.0, rel=2e-3)
    assert lam_w == pytest.approx(lam_u, rel=2e-3)


def test_paper_literal_normalisation_doubles_the_rate():
    """Z b^2 of Eq. Kij read literally for FCC (Z = 12 nearest neighbours, b = a/sqrt2:
    Z b^2 = 6 a^2) against the default second moment of the 18-neighbour shell
    (S2 = 12 a^2): K doubles, so a sin mode decays at twice the lattice-sum rate."""
    a = I.CU_A
    x = I.fcc_lattice(10, 3, 3, a)
    box = np.array([10 * a, 3 * a, 3 * a])
    per = np.array([1, 1, 1], dtype=np.int32)
    rowptr, col = oracle.neighbors(x, box, per, 4.0)
    k = 2 * math.pi / (10 * a)
    basis = np.sin(k * x[:, 0])
    T0, amp, dt, n = 300.0, 1e-4, 1e-4, 50
    zeros = np.zeros(x.shape[0])
    rates = []
    for zb2 in (I.fcc_shell_s2(a, 4.0), 6.0 * a * a):
        K = 2.0 * 3 * 400.0 / (96.6 * 300.0 * zb2 * 1e-20) * 1e-15
        T = T0 + amp * basis
        oracle.substeps(rowptr, col, T, zeros, np.zeros(x.shape[0], np.uint8), zeros.copy(), n, dt, 1e5, K,
                        0.0, 0.0)
        a1 = float((T - T0) @ basis / (basis @ basis))
        # explicit Euler: the mode's factor per substep is 1 - dt lambda exactly
        rates.append((1.0 - (a1 / amp) ** (1.0 / n)) / dt)
    assert I.fcc_shell_s2(a, 4.0) == pytest.approx(12 * a * a, rel=1e-12)
    assert rates[1] == pytest.approx(2.0 * rates[0], rel=1e-5)
