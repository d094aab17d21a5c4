"""Pins of the oracle's laser source term (Sec. 5, Eq. LaserIntesity).

The absorbed power density of a Gaussian pulse decaying below the irradiated
surface is

    S(d, t) = (F / l_p) exp(-d / l_p) exp(-(t - t0)^2 / (2 s^2)) / (s sqrt(2 pi)),

with F the absorbed fluence, l_p the penetration depth, d the depth below the
initial top surface and s the pulse's standard deviation, s = FWHM / (2 sqrt(2 ln 2)).
It raises T_e at the rate S / C_e, and the energy it brings in over the whole
pulse is V_atom (F / l_p) exp(-d / l_p) per atom.

Every expected value below is computed here from the workload's numbers in the
units the workload states them in (fluence in J/cm^2, depth scale in nm, pulse
width as a FWHM in fs), with SI conversions written out in this file, so that a
wrong unit factor, l_p taken in the wrong unit, or the FWHM used as the standard
deviation fails a test.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1810_12357_gb300 import inputs as I

# the laser-slab workload as stated: 0.1 J/cm^2 absorbed, 15 nm, 100 fs FWHM, peak at 50 fs
FLUENCE_J_PER_CM2 = 0.1
LP_NM = 15.0
FWHM_FS = 100.0
T0_FS = 50.0

J_PER_EV = 1.602176634e-19


def _sigma_fs(fwhm_fs: float) -> float:
    # half maximum of exp(-t^2 / (2 s^2)) at t = FWHM / 2  =>  s = FWHM / sqrt(8 ln 2)
    return fwhm_fs / math.sqrt(8.0 * math.log(2.0))


def _power_density_W_m3(depth_A, t_fs, fluence_J_cm2=FLUENCE_J_PER_CM2, lp_nm=LP_NM):
    """S(d, t) in W m^-3, from the workload's own units."""
    F = fluence_J_cm2 * 1.0e4                     # J/cm^2 -> J/m^2
    lp = lp_nm * 1.0e-9                           # nm -> m
    s = _sigma_fs(FWHM_FS) * 1.0e-15              # fs -> s
    d = np.asarray(depth_A, dtype=np.float64) * 1.0e-10
    tt = (t_fs - T0_FS) * 1.0e-15
    return (F / lp) * np.exp(-d / lp) * math.exp(-tt * tt / (2.0 * s * s)) / (s * math.sqrt(2.0 * math.pi))


def _source(fluence_J_cm2=FLUENCE_J_PER_CM2):
    src = dict(I.params_laser()["laser"])
    src["fluence_Jm2"] *= fluence_J_cm2 / FLUENCE_J_PER_CM2
    return src


def test_workload_pulse_is_the_stated_one():
    las = I.params_laser()["laser"]
    s = las["sigma_fs"]
    # the Gaussian in time is at half its maximum FWHM / 2 away from its peak
    assert math.exp(-0.5 * (0.5 * FWHM_FS / s) ** 2) == pytest.approx(0.5, rel=1e-14)
    assert las["t0_fs"] == T0_FS
    assert las["fluence_Jm2"] == pytest.approx(FLUENCE_J_PER_CM2 * 1.0e4, rel=1e-15)
    assert las["lp_A"] == pytest.approx(LP_NM * 10.0, rel=1e-15)
    # one FWHM is 2.3548 standard deviations
    assert FWHM_FS / s == pytest.approx(2.0 * math.sqrt(2.0 * math.log(2.0)), rel=1e-15)


@pytest.mark.parametrize("t_fs", [T0_FS, T0_FS - 42.0, T0_FS + 106.0, 0.0])
def test_one_substep_raises_T_by_S_over_Ce(t_fs):
    # no pair terms (empty rows), no coupling: a substep changes T_i by dt S_i / C_e only
    depth = np.array([0.0, 3.615, 75.0, 150.0, 300.0, 722.0])
    n = depth.shape[0]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(0, dtype=np.int32)
    T = np.full(n, 300.0)
    T0 = T.copy()
    A = np.zeros(n)
    chi = np.zeros(n, dtype=np.uint8)
    Ce = 3.5e6                  # J m^-3 K^-1
    V = I.CU_A ** 3 / 4.0       # A^3
    dt = 1.0e-3                 # fs
    st, esrc = oracle.substeps(rowptr, col, T, np.full(n, 300.0), chi, A, 1, dt, 1.0e5, 0.0, 0.0, 0.0,
                               depth=depth, source=_source(), Ce_SI=Ce, vatom_A3=V, t_start=t_fs)
    assert st == 1
    S = _power_density_W_m3(depth, t_fs)
    dT_expected = S / Ce * (dt * 1.0e-15)               # K
    assert np.allclose(T - T0, dT_expected, rtol=1e-9, atol=0.0)
    # the energy the source brought in this substep: sum_i S_i V_atom dt
    e_expected = float(S.sum()) * V * 1.0e-30 * dt * 1.0e-15 / J_PER_EV
    assert esrc == pytest.approx(e_expected, rel=1e-12)
    # exponential attenuation with depth: one l_p deeper is e times weaker
    i150 = 3
    assert (T[0] - 300.0) / (T[i150] - 300.0) == pytest.approx(math.e, rel=1e-9)


def test_energy_of_the_whole_pulse_is_the_fluence_integral():
    # E_src over t0 +- 6 s equals sum_i V (F / l_p) e^{-d_i / l_p} times the pulse
    # fraction 1/2 [erf(u1) - erf(u0)] (u = (t - t0) / (s sqrt 2)); the substep sum
    # is a left Riemann sum of a smooth pulse, exact to far below the tolerance here
    depth = np.linspace(0.0, 900.0, 41)
    n = depth.shape[0]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(0, dtype=np.int32)
    T = np.full(n, 300.0)
    A = np.zeros(n)
    chi = np.zeros(n, dtype=np.uint8)
    V = I.CU_A ** 3 / 4.0
    s = _sigma_fs(FWHM_FS)
    t_start, dt = T0_FS - 6.0 * s, 0.25
    n_sub = int(round(12.0 * s / dt))
    t_end = t_start + n_sub * dt
    st, esrc = oracle.substeps(rowptr, col, T, np.full(n, 300.0), chi, A, n_sub, dt, 1.0e9, 0.0, 0.0, 0.0,
                               depth=depth, source=_source(), Ce_SI=1.0e9, vatom_A3=V, t_start=t_start)
    assert st == n_sub
    F = FLUENCE_J_PER_CM2 * 1.0e4
    lp = LP_NM * 1.0e-9
    frac = 0.5 * (math.erf((t_end - T0_FS) / (s * math.sqrt(2.0)))
                  - math.erf((t_start - T0_FS) / (s * math.sqrt(2.0))))
    per_atom = (F / lp) * np.exp(-depth * 1.0e-10 / lp) * V * 1.0e-30 / J_PER_EV    # eV per whole pulse
    assert frac > 1.0 - 2.0e-9
    assert esrc == pytest.approx(float(per_atom.sum()) * frac, rel=1e-9)


def test_slab_without_coupling_gains_exactly_the_pulse_energy():
    # a slab with free z surfaces, vacancies, conduction on, no electron-phonon
    # coupling, frozen atoms: over the whole pulse its electrons gain the fluence
    # integral over its atoms, while conduction moves the heat inward
    s = I.laser_slab_system(3, 8, 7)
    fl = 0.001                                       # J/cm^2: keeps theta inside [0, 1]
    p = dict(I.params_laser(), G=0.0, couple_mode=0, frozen=1, kappa_mode=0, kappa0=0.4,
             flux_prec=1, dt_sub=0.5, laser=_source(fl))
    sim = oracle.OracleSim(p, s.box, s.periodic, s.mass_amu, s.type, depth=s.depth)
    sim.set_te(s.Te)
    sig = _sigma_fs(FWHM_FS)
    t_start = T0_FS - 6.0 * sig
    n_sub = int(round(12.0 * sig / p["dt_sub"]))
    sim.build(s.x, s.v)
    assert sim.stability < 2.0
    sim.substeps(n_sub, t_start=t_start)
    t_end = t_start + n_sub * p["dt_sub"]
    e = sim.energy()
    z_top = s.x[:, 2].max()
    d = (z_top - s.x[:, 2]) * 1.0e-10                 # depth below the initial top surface [m]
    lp = LP_NM * 1.0e-9
    frac = 0.5 * (math.erf((t_end - T0_FS) / (sig * math.sqrt(2.0)))
                  - math.erf((t_start - T0_FS) / (sig * math.sqrt(2.0))))
    V = I.CU_A ** 3 / 4.0
    expected = float((fl * 1.0e4 / lp * np.exp(-d / lp)).sum()) * V * 1.0e-30 / J_PER_EV * frac
    assert e["E_src"] == pytest.approx(expected, rel=1e-9)
    assert e["E_e"] - e["E_e0"] == pytest.approx(expected, rel=1e-9)
    assert e["E_lat"] == 0.0
    # conduction moved heat inward: against the source alone (dT_i = its absorbed
    # energy density / C_e), the top layer ends cooler and the bottom layer warmer
    dT_src = fl * 1.0e4 / lp * np.exp(-d / lp) * frac / sim.Ce
    dT = sim.T - s.Te
    top, bottom = d < 1.0e-10, d > d.max() - 1.0e-10
    assert np.all(dT[top] < dT_src[top]) and np.all(dT[bottom] > dT_src[bottom])
