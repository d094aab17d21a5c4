"""Pins of the oracle's fixed-temperature border (a Dirichlet condition on T_e,
the 300 K border shell of the paper's cascade runs, Sec. 5): an empty border is
the plain method, the border keeps the energy balance exactly, a slab between
two fixed layers relaxes to the root of the algebraic steady-state equations
F_i(T) = 0 of its free atoms (solved here without the time stepping), and the
MD-step ledger closes with the coupling on."""
import numpy as np
import pytest

import oracle
from paper_1810_12357_gb300 import inputs as I


def _slab(nx=10, ny=3, nz=3):
    a = I.CU_A
    x = I.fcc_lattice(nx, ny, nz, a)
    box = np.array([nx * a, ny * a, nz * a])
    per = np.array([1, 1, 1], dtype=np.int32)
    rowptr, col = oracle.neighbors(x, box, per, 4.0)
    return a, x, box, per, rowptr, col


def _run(rowptr, col, T, n_sub, K, Tfix=None, eres=None, dt=1e-3, Tmax=1e5):
    n = T.shape[0]
    zeros = np.zeros(n)
    st, _ = oracle.substeps(rowptr, col, T, zeros, np.zeros(n, np.uint8), zeros.copy(), n_sub, dt, Tmax, K,
                            0.0, 0.0, Tfix=Tfix, eres=eres)
    assert st == n_sub
    return T


def test_empty_border_is_the_plain_method():
    a, x, box, per, rowptr, col = _slab()
    rng = np.random.default_rng(0)
    T0 = 300.0 + 200.0 * rng.random(x.shape[0])
    Ta = _run(rowptr, col, T0.copy(), 50, 40.0)
    eres = np.zeros(1)
    Tb = _run(rowptr, col, T0.copy(), 50, 40.0, Tfix=np.full(x.shape[0], np.nan), eres=eres)
    assert np.array_equal(Ta, Tb)
    assert eres[0] == 0.0


def test_border_keeps_the_energy_balance():
    # coupling off: the pair fluxes are odd, so sum_i T_i changes only by what the
    # border absorbs
    a, x, box, per, rowptr, col = _slab()
    rng = np.random.default_rng(1)
    T0 = 300.0 + 500.0 * rng.random(x.shape[0])
    Tfix = np.where(x[:, 0] < a, 600.0, np.nan)
    T0[x[:, 0] < a] = 600.0
    eres = np.zeros(1)
    T = _run(rowptr, col, T0.copy(), 400, 40.0, Tfix=Tfix, eres=eres)
    assert np.all(T[x[:, 0] < a] == 600.0)
    assert abs(T.sum() + eres[0] - T0.sum()) < 1e-11 * T0.sum()
    assert abs(eres[0]) > 1.0        # the border did exchange energy


def test_slab_relaxes_to_the_algebraic_steady_state():
    from scipy.optimize import root
    a, x, box, per, rowptr, col = _slab()
    n = x.shape[0]
    Tmax, K, dt = 1e5, 40.0, 1e-3     # dt 36 K = 1.44 < 2
    hot = x[:, 0] < a
    cold = (x[:, 0] >= 5 * a) & (x[:, 0] < 6 * a)
    Tfix = np.full(n, np.nan)
    Tfix[hot] = 900.0
    Tfix[cold] = 300.0
    free = ~(hot | cold)
    T = np.where(hot, 900.0, 300.0).astype(np.float64)
    eres = np.zeros(1)
    # relax; then the free atoms' pair-flux sums vanish
    T = _run(rowptr, col, T, 60000, K, Tfix=Tfix, eres=eres, dt=dt, Tmax=Tmax)

    def resid(Tf):
        full = Tfix.copy()
        full[free] = Tf
        return oracle.flux_sum(rowptr, col, full / Tmax)[free] * 1e3

    sol = root(resid, np.full(free.sum(), 600.0), method="hybr", tol=1e-12)
    Ts = sol.x
    assert np.max(np.abs(resid(Ts))) < 1e-9    # a root to rounding (the solver may stop at its xtol)
    err = np.max(np.abs(T[free] - Ts))
    print(f"slab steady state: max |T - root| = {err:.3e} K, range {Ts.min():.2f}..{Ts.max():.2f} K")
    assert err < 1e-6
    # the profile runs between the two border temperatures
    assert 300.0 < Ts.min() and Ts.max() < 900.0 and Ts.max() - Ts.min() > 300.0
    # in the steady state the hot layer feeds exactly what the cold one absorbs
    F = oracle.flux_sum(rowptr, col, T / Tmax)
    assert abs(F[hot].sum() + F[cold].sum()) < 1e-9 * np.abs(F[hot]).sum()


@pytest.mark.parametrize("couple_mode", [0, 1])
def test_ledger_closes_with_border_and_coupling(couple_mode):
    s = I.hot_spot_system(6, 4, peak=4000.0)
    p = dict(I.params_hotspot_fp64(), couple_mode=couple_mode, G=3e18, frozen=0)
    sim = oracle.OracleSim(p, s.box, s.periodic, s.mass_amu, s.type)
    T0 = s.Te.copy()
    edge = np.any((s.x < 3.0) | (s.x > s.box - 3.0), axis=1)
    Tfix = np.where(edge, 300.0, np.nan)
    T0[edge] = 300.0
    sim.set_te(T0)
    sim.set_border(Tfix)
    x, v = s.x.copy(), s.v.copy()
    for step in range(3):
        sim.build(x, v)
        sim.substeps(40)
        sim.couple(v, 40 * p["dt_sub"])
    e = sim.energy()
    assert np.all(sim.T[edge] == 300.0)
    assert e["E_res"] > 0.0            # heat from the hot spot reached the border
    assert abs(e["drift"]) < 1e-12
