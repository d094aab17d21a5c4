"""Pins of the oracle's LOCAL per-atom C_e / kappa_e form (oracle_substeps_local):
C_e,i = min(gamma T_i, cap), kappa_i = kappa0 T_i / T_lat (or kappa0), pair energy
rates with kappa_ij = (kappa_i + kappa_j) / 2, each atom's electron energy density
U(T) = int_0^T C_e advanced explicitly and T recovered by inverting U.

What fixes it, independently of its own formula:
  * sum_i U(T_i) is conserved exactly (pair energy rates are antisymmetric);
  * an isolated periodic lattice relaxes to the uniform T with U(T) = mean U(T_i),
    not to the mean temperature (closed form, below and across the cap);
  * a small sin mode decays at c(theta) K sum_j (1 - cos k.r_j) with
    K = 2 d kappa0 / (gamma S2 T_lat) (kappa_mode 1): the lattice sum, and the
    global form's rate when <T_e> is the background;
  * with the pair terms off, T follows the closed form of
    gamma T dT/dt = -G (T - T_l), to first order in dt;
  * above the cap with constant kappa every C_e,i is the cap: the global form
    (oracle_substeps, pinned on its own) with C_e = cap, to rounding."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_1810_12357_gb300 import inputs as I

GAMMA = 96.6
KB_J = 1.380649e-23
EV_J = 1.602176634e-19


def _lattice(nx=4, ny=3, nz=3, disp=0.0, seed=0):
    a = I.CU_A
    x = I.fcc_lattice(nx, ny, nz, a)
    box = np.array([nx * a, ny * a, nz * a])
    if disp > 0:
        x = I.wrap(x + np.random.default_rng(seed).normal(0, disp, x.shape), box, np.array([1, 1, 1]))
    per = np.array([1, 1, 1], dtype=np.int32)
    rowptr, col = oracle.neighbors(x, box, per, 4.0)
    return a, x, box, rowptr, col


def _cap(a):
    """3 k_B per atomic volume a^3 / 4 [J m^-3 K^-1]."""
    return 3.0 * KB_J / (a ** 3 / 4.0 * 1e-30)


def _U(T, cap):
    return np.array([oracle.ce_energy(t, GAMMA, cap) for t in np.atleast_1d(T)])


def _run(rowptr, col, T, n_sub, dt, *, kappa_mode=1, kappa0=400.0, Tlat=300.0, cap=0.0, G=0.0, Tl=None,
         chi=None, Tmax=1.0e5, vatom=None, weights=None):
    n = T.shape[0]
    a = I.CU_A
    Tl = np.zeros(n) if Tl is None else Tl
    chi = np.zeros(n, np.uint8) if chi is None else chi
    A = np.zeros(n)
    st, _, _ = oracle.substeps_local(rowptr, col, T, Tl, chi, A, n_sub, dt, Tmax, kappa0=kappa0,
                                     kappa_mode=kappa_mode, Tlat=Tlat, dim_d=3,
                                     S2_A2=I.fcc_shell_s2(a, 4.0), gamma=GAMMA, cap_SI=cap, G=G,
                                     vatom_A3=vatom if vatom else a ** 3 / 4.0, weights=weights)
    return st, A


@pytest.mark.parametrize("kappa_mode,lo,hi,capped", [(1, 300.0, 3000.0, False), (0, 300.0, 3000.0, False),
                                                     (1, 20000.0, 60000.0, True)])
def test_local_form_conserves_the_electron_energy(kappa_mode, lo, hi, capped):
    a, x, box, rowptr, col = _lattice(disp=0.08, seed=5)
    cap = _cap(a) if capped else 0.0
    rng = np.random.default_rng(2)
    T = lo + (hi - lo) * rng.random(x.shape[0])
    U0 = _U(T, cap).sum()
    T0 = T.copy()
    # K = 2 d kappa0 / (gamma S2 T_lat) = 52.8 / fs at T_lat = 300 K (87 / fs for the
    # capped set): dt (2 n_max K) stays below 2
    st, _ = _run(rowptr, col, T, 200, 2e-4, kappa_mode=kappa_mode, cap=cap)
    assert st == 200
    assert np.max(np.abs(T - T0)) > 1.0
    assert abs(_U(T, cap).sum() - U0) < 2e-14 * U0 * math.sqrt(200)
    # ... while the temperature sum is not conserved (C_e differs from atom to atom)
    assert abs(T.sum() - T0.sum()) > 1e-6 * T0.sum()


@pytest.mark.parametrize("lo,hi,capped", [(300.0, 3000.0, False), (20000.0, 60000.0, True)])
def test_isolated_lattice_relaxes_to_the_mean_energy(lo, hi, capped):
    a, x, box, rowptr, col = _lattice()
    cap = _cap(a) if capped else 0.0
    rng = np.random.default_rng(9)
    T = lo + (hi - lo) * rng.random(x.shape[0])
    # the end state: one temperature whose energy density is the mean one
    Uinf = _U(T, cap).mean()
    Tinf = oracle.ce_energy_inv(Uinf, GAMMA, cap)
    if capped:
        Tc = cap / GAMMA
        assert T.min() < Tc < T.max()
        # piecewise closed form, written out here
        Uc = 0.5 * cap * Tc
        assert Tinf == pytest.approx(Tc + (Uinf - Uc) / cap if Uinf > Uc else math.sqrt(2 * Uinf / GAMMA), rel=1e-14)
    else:
        assert Tinf == pytest.approx(math.sqrt(np.mean(T * T)), rel=1e-13)
    assert abs(Tinf - T.mean()) > 0.01 * T.mean()
    st, _ = _run(rowptr, col, T, 1500, 4e-4, cap=cap)
    assert st == 1500
    assert np.max(np.abs(T - Tinf)) < 1e-9 * Tinf


def _mode(kappa_mode, T0, Tlat, n_sub, dt, amp=1e-4, ncx=10):
    a = I.CU_A
    x = I.fcc_lattice(ncx, 3, 3, a)
    box = np.array([ncx * a, 3 * a, 3 * a])
    per = np.array([1, 1, 1], dtype=np.int32)
    rowptr, col = oracle.neighbors(x, box, per, 4.0)
    k = 2 * math.pi / (ncx * a)
    basis = np.sin(k * x[:, 0])
    T = T0 + amp * basis
    a0 = float((T - T0) @ basis / (basis @ basis))
    st, _ = _run(rowptr, col, T, n_sub, dt, kappa_mode=kappa_mode, Tlat=Tlat)
    assert st == n_sub
    a1 = float((T - T0) @ basis / (basis @ basis))
    th = T0 / 1.0e5
    c = 1 - 2 * th * (1 - th)
    shell = I.fcc_shell_vectors(a, 4.0)
    S2 = I.fcc_shell_s2(a, 4.0)
    geo = 2.0 * 3 / (S2 * 1e-20)
    K = geo * 400.0 / (GAMMA * (Tlat if kappa_mode == 1 else T0)) * 1e-15
    lam = c * K * float((1 - np.cos(k * shell[:, 0])).sum())
    return a0, a1, lam, rowptr, col, K, x, k


@pytest.mark.parametrize("kappa_mode,T0,Tlat", [(1, 300.0, 300.0), (1, 2000.0, 450.0), (0, 1500.0, 300.0)])
def test_small_mode_decays_at_the_lattice_sum(kappa_mode, T0, Tlat):
    n, dt, amp = 100, 5e-4, 1e-4
    a0, a1, lam, rowptr, col, K, x, k = _mode(kappa_mode, T0, Tlat, n, dt, amp)
    assert a1 == pytest.approx(a0 * (1 - dt * lam) ** n, rel=2e-6)
    # the global form (oracle_substeps) at <T_e> = T0, C_e = gamma T0 and
    # kappa_e = kappa0 T0 / T_lat (mode 1) or kappa0, gives the same mode
    basis = np.sin(k * x[:, 0])
    T = T0 + amp * basis
    nn = T.shape[0]
    kap = 400.0 * (T0 / Tlat if kappa_mode == 1 else 1.0)
    Kg = 2.0 * 3 * kap / (GAMMA * T0 * I.fcc_shell_s2(I.CU_A, 4.0) * 1e-20) * 1e-15
    oracle.substeps(rowptr, col, T, np.zeros(nn), np.zeros(nn, np.uint8), np.zeros(nn), n, dt, 1.0e5, Kg, 0.0, 0.0)
    ag = float((T - T0) @ basis / (basis @ basis))
    assert ag == pytest.approx(a1, rel=2e-6)


def test_coupling_follows_the_closed_form():
    """gamma T dT/dt = -G (T - T_l): t(T) = (gamma/G) [(T0 - T) + T_l ln((T0 - T_l)/(T - T_l))]."""
    a, x, box, rowptr, col = _lattice(nx=2, ny=2, nz=2)
    n = x.shape[0]
    G, Tl0, T0, t_end = 1.0e17, 300.0, 5000.0, 2000.0     # W m^-3 K^-1, K, K, fs
    tau = GAMMA / G * 1e15                                   # fs per kelvin of gamma T / G

    def t_of(T):
        return tau * ((T0 - T) + Tl0 * math.log((T0 - Tl0) / (T - Tl0)))

    T_exact = brentq(lambda T: t_of(T) - t_end, Tl0 + 1e-9, T0)
    errs = []
    for dt in (2.0, 1.0, 0.5):
        T = np.full(n, T0)
        st, A = _run(rowptr, col, T, int(round(t_end / dt)), dt, kappa0=0.0, kappa_mode=0, G=G,
                     Tl=np.full(n, Tl0), chi=np.ones(n, np.uint8))
        assert st > 0
        assert np.all(T == T[0])
        errs.append(abs(T[0] - T_exact))
        # the energy the lattice received is exactly what the electrons lost
        vat = a ** 3 / 4.0 * 1e-30
        lost = (oracle.ce_energy(T0, GAMMA, 0.0) - oracle.ce_energy(T[0], GAMMA, 0.0)) * vat / EV_J
        assert A.sum() == pytest.approx(n * lost, rel=1e-12)
    assert errs[-1] < 2e-4 * T_exact
    # first order in dt
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


def test_above_the_cap_with_constant_kappa_is_the_global_form():
    a, x, box, rowptr, col = _lattice(disp=0.05, seed=1)
    n = x.shape[0]
    cap = _cap(a)
    rng = np.random.default_rng(4)
    T = 40000.0 + 20000.0 * rng.random(n)
    Tl = 300.0 + 100.0 * rng.random(n)
    chi = (rng.random(n) < 0.8).astype(np.uint8)
    G, Tmax, dt = 2.0e17, 1.0e5, 2e-3
    Tg, Ag = T.copy(), np.zeros(n)
    S2 = I.fcc_shell_s2(a, 4.0)
    vatom = a ** 3 / 4.0
    K = 2.0 * 3 * 400.0 / (cap * S2 * 1e-20) * 1e-15
    st_g = oracle.substeps(rowptr, col, Tg, Tl, chi, Ag, 60, dt, Tmax, K, G / cap * 1e-15,
                           G * vatom * 1e-30 / EV_J * 1e-15)[0]
    st, A = _run(rowptr, col, T, 60, dt, kappa_mode=0, cap=cap, G=G, Tl=Tl, chi=chi, Tmax=Tmax)
    assert st == st_g == 60
    assert T.min() > cap / GAMMA
    assert np.max(np.abs(T - Tg)) < 1e-12 * Tg.max()
    assert np.max(np.abs(A - Ag)) < 1e-12 * np.abs(Ag).max()


def test_local_weights_multiply_the_pair_rates():
    """Uniform weights 1 are the unweighted form; weights 2 double the pair rates
    (one substep, coupling off)."""
    a, x, box, rowptr, col = _lattice(disp=0.05, seed=6)
    rng = np.random.default_rng(8)
    T = 300.0 + 3000.0 * rng.random(x.shape[0])
    ones = np.ones(col.shape[0])
    Ta, Tb, Tc = T.copy(), T.copy(), T.copy()
    _run(rowptr, col, Ta, 1, 1e-4)
    _run(rowptr, col, Tb, 1, 1e-4, weights=ones)
    _run(rowptr, col, Tc, 1, 1e-4, weights=2.0 * ones)
    assert np.array_equal(Ta, Tb)
    Ua, Uc, U0 = _U(Ta, 0.0), _U(Tc, 0.0), _U(T, 0.0)
    assert np.allclose(Uc - U0, 2.0 * (Ua - U0), rtol=1e-9, atol=1e-12 * U0.max())


@pytest.mark.parametrize("couple_mode", [0, 1])
def test_local_ledger_closes_with_coupling(couple_mode):
    s = I.hot_spot_system(6, 4, peak=4000.0)
    p = dict(I.params_hotspot_fp64(), couple_mode=couple_mode, G=3e18, frozen=0, ce_mode=1, kappa_mode=1)
    sim = oracle.OracleSim(p, s.box, s.periodic, s.mass_amu, s.type)
    sim.set_te(s.Te)
    x, v = s.x.copy(), s.v.copy()
    for step in range(3):
        sim.build(x, v)
        assert sim.stability < 2.0
        sim.substeps(40)
        sim.couple(v, 40 * p["dt_sub"])
    e = sim.energy()
    assert e["E_lat"] != 0.0
    assert abs(e["drift"]) < 1e-12


def test_local_border_keeps_the_energy_balance():
    s = I.hot_spot_system(6, 4, peak=4000.0)
    p = dict(I.params_hotspot_fp64(), couple_mode=0, G=3e18, frozen=0, ce_mode=1, kappa_mode=0)
    sim = oracle.OracleSim(p, s.box, s.periodic, s.mass_amu, s.type)
    T0 = s.Te.copy()
    edge = np.any((s.x < 3.0) | (s.x > s.box - 3.0), axis=1)
    T0[edge] = 300.0
    sim.set_te(T0)
    sim.set_border(np.where(edge, 300.0, np.nan))
    x, v = s.x.copy(), s.v.copy()
    for step in range(3):
        sim.build(x, v)
        sim.substeps(40)
        sim.couple(v, 40 * p["dt_sub"])
    e = sim.energy()
    assert np.all(sim.T[edge] == 300.0)
    assert e["E_res"] > 0.0
    assert abs(e["drift"]) < 1e-12
