"""The 1-D nickel bar of Sec. 3.1: master-equation electrons (Eq. HeatTransport)
coupled to a lattice solved by a three-point finite-difference Fourier law
(second line of Eq. 1d_FE), forward Euler, periodic.

Pins the oracle's substep (flux plus the G term and the energy it hands over)
against a closed form that follows from energy conservation alone: the final
common temperature  T_eq = (C_e sum T_e0 + rho C_l sum T_l0) / (N (C_e + rho C_l)).
"""
import math

import numpy as np
import pytest

import oracle

# Sec. 3.1 parameters
A0 = 3.562                    # lattice constant of Ni [A]
N_SITES = 141                 # 100 a0 / (a0 / sqrt 2) = 141.4 -> 141 sites on the ring
B = 100.0 * A0 / N_SITES      # site spacing [A]
G = 3.6e17                    # W m^-3 K^-1
CE = 3.6886e5                 # J m^-3 K^-1 (constant in this test, as in the paper's FD run)
KAPPA = 91.0                  # W m^-1 K^-1
KAPPA_L = 0.05 * KAPPA
RHO_CL = 8890.0 * 400.0       # J m^-3 K^-1
DT = 0.1                      # fs
TMAX = 2.0e4


def _ring():
    n = N_SITES
    rowptr = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
    col = np.empty(2 * n, dtype=np.int32)
    for i in range(n):
        lo, hi = sorted(((i - 1) % n, (i + 1) % n))
        col[2 * i], col[2 * i + 1] = lo, hi
    return rowptr, col


def _initial():
    x = np.arange(N_SITES) * B
    Te = np.full(N_SITES, 300.0)
    hot = np.abs(x - x[N_SITES // 2]) <= A0   # span 2 a0 at the centre
    Te[hot] = 6000.0
    return Te, np.full(N_SITES, 300.0), int(hot.sum())


def _run(t_end_fs, sub_per_lattice=10, electrons="master"):
    rowptr, col = _ring()
    Te, Tl, n_hot = _initial()
    K = 2 * 1 * KAPPA / (CE * 2 * (B * 1e-10) ** 2) * 1e-15   # Eq. Kij with d = 1, Z = 2 [1/fs]
    cG = G / CE * 1e-15
    VG = G * 1e-15                # per unit volume: A is J m^-3 here
    chi = np.ones(N_SITES, dtype=np.uint8)
    A = np.zeros(N_SITES)
    dt_l = DT * sub_per_lattice
    Dl = KAPPA_L / RHO_CL * 1e20 * 1e-15 / B ** 2    # lattice diffusion number per fs
    De = KAPPA / CE * 1e20 * 1e-15 / B ** 2
    inv0 = CE * Te.sum() + RHO_CL * Tl.sum()
    n_iter = int(round(t_end_fs / dt_l))
    for it in range(n_iter):
        if electrons == "master":
            st, _ = oracle.substeps(rowptr, col, Te, Tl, chi, A, sub_per_lattice, DT, TMAX, K, cG, VG)
            assert st == sub_per_lattice
        else:   # Fourier law for the electrons too (first line of Eq. 1d_FE)
            for s in range(sub_per_lattice):
                lap = np.roll(Te, 1) + np.roll(Te, -1) - 2 * Te
                d = Te - Tl
                A += DT * VG * d
                Te = Te + DT * (De * lap - cG * d)
        lapl = np.roll(Tl, 1) + np.roll(Tl, -1) - 2 * Tl
        Tl = Tl + dt_l * Dl * lapl + A / RHO_CL
        A[:] = 0.0
    inv1 = CE * Te.sum() + RHO_CL * Tl.sum()
    return Te, Tl, inv0, inv1, n_hot, K


def test_two_bath_equilibrium_closed_form():
    Te, Tl, inv0, inv1, n_hot, K = _run(60000.0, sub_per_lattice=20)
    assert K * DT == pytest.approx(0.3866, abs=1e-3)    # stable: dt * 4K = 1.55 < 2
    assert abs(inv1 - inv0) / inv0 < 1e-12
    T_eq = 300.0 + n_hot * 5700.0 * CE / (N_SITES * (CE + RHO_CL))
    assert n_hot == 3 and T_eq == pytest.approx(311.3976, abs=1e-3)
    # the conserved combination fixes T_eq exactly; after 60 ps both fields sit on it
    assert (CE * Te.mean() + RHO_CL * Tl.mean()) / (CE + RHO_CL) == pytest.approx(T_eq, rel=1e-12)
    assert np.abs(Te - T_eq).max() < 5e-3
    assert np.abs(Tl - T_eq).max() < 5e-3


def test_master_equation_tracks_fourier_electrons():
    # The paper reports the two electron models agree up to small differences
    # (long-wave origin of Eq. Kij, c(theta) = 1 - 2 theta (1 - theta)); record the gap.
    Te_m, Tl_m, *_ = _run(3000.0)
    Te_f, Tl_f, *_ = _run(3000.0, electrons="fourier")
    rise = Te_f.max() - 300.0
    assert np.abs(Te_m - Te_f).max() < 0.1 * rise
    assert np.abs(Tl_m - Tl_f).max() < 0.1 * (Tl_f.max() - 300.0)
