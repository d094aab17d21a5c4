"""Pins of the oracle's lattice side: shifted-force Morse forces (oracle_forces),
the velocity-Verlet kick, and electronic stopping in the hand-over.

  * F = -grad E, by central differences on the position grid, for a displaced
    lattice with pairs near the cutoff;
  * sum_i F_i = 0 (Newton's third law);
  * perfect FCC: F = 0 and E_i = (12 phi_sf(a / sqrt 2) + 6 phi_sf(a)) / 2;
  * phi_sf and phi_sf' vanish at the cutoff (energy continuous as a pair leaves);
  * a velocity-Verlet run conserves KE + PE to O(dt^2): halving dt divides the
    energy error by about 4;
  * stopping above the cut removes K (1 - exp(-2 beta dt)) from a fast atom's
    kinetic energy and gives exactly that to its electrons; below the cut nothing."""
import math

import numpy as np
import pytest

import oracle
from paper_1810_12357_gb300 import inputs as I

D, ALPHA, R0, RC = 0.3429, 1.3588, 2.866, 4.0      # Cu, Girifalco and Weizer
MVV = 1.66053906660e-27 * 1.0e10 / 1.602176634e-19


def _cell(nx=4, ny=3, nz=3, disp=0.0, seed=0, a=I.CU_A):
    x = I.fcc_lattice(nx, ny, nz, a)
    box = np.array([nx * a, ny * a, nz * a])
    per = np.array([1, 1, 1], dtype=np.int32)
    if disp > 0:
        x = I.wrap(x + np.random.default_rng(seed).normal(0, disp, x.shape), box, per)
    return x, box, per


def _fe(x, box, per):
    rowptr, col = oracle.neighbors(x, box, per, RC)
    return oracle.forces(x, box, per, rowptr, col, D=D, alpha=ALPHA, r0=R0, rc=RC)


def _phi_sf(r):
    pc, dpc = oracle.morse(RC, D, ALPHA, R0)
    ph, _ = oracle.morse(r, D, ALPHA, R0)
    return ph - pc - (r - RC) * dpc


def test_forces_are_minus_the_energy_gradient():
    x, box, per = _cell(disp=0.12, seed=3)
    F, E = _fe(x, box, per)
    h = 64.0 / 1048576.0          # 64 grid steps: positions stay on the quantisation grid
    rng = np.random.default_rng(1)
    for i in rng.choice(x.shape[0], 6, replace=False):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            # the neighbour lists must not change between the two positions
            _, Ep = _fe(xp, box, per)
            _, Em = _fe(xm, box, per)
            g = (Ep.sum() - Em.sum()) / (2 * h)
            assert F[i, k] == pytest.approx(-g, abs=2e-6 * max(1.0, abs(g)))


def test_newton_third_law_and_the_perfect_lattice():
    x, box, per = _cell(disp=0.1, seed=4)
    F, _ = _fe(x, box, per)
    assert np.max(np.abs(F.sum(axis=0))) < 1e-12 * np.abs(F).sum()
    # a lattice constant whose half lies on the 2^-20 A position grid: the
    # quantised lattice is then exactly the perfect one
    a = round(I.CU_A * 2 ** 19) / 2 ** 19
    xp, boxp, perp = _cell(a=a)
    Fp, Ep = _fe(xp, boxp, perp)
    assert np.max(np.abs(Fp)) < 1e-12
    e_shell = 0.5 * (12 * _phi_sf(a / math.sqrt(2)) + 6 * _phi_sf(a))
    assert np.allclose(Ep, e_shell, rtol=1e-12, atol=0)


def test_shifted_force_vanishes_at_the_cutoff():
    pc, dpc = oracle.morse(RC, D, ALPHA, R0)
    assert _phi_sf(RC) == 0.0
    # phi_sf' = phi' - phi'(rc): central difference of phi_sf at rc from inside
    h = 1e-6
    assert abs((_phi_sf(RC) - _phi_sf(RC - h)) / h) < 1e-5
    # the Morse minimum: phi(r0) = -D, phi'(r0) = 0
    p0, d0 = oracle.morse(R0, D, ALPHA, R0)
    assert p0 == pytest.approx(-D, rel=1e-15) and d0 == 0.0


def _nve(dt, n_steps, x, v, box, per, mass):
    x, v = x.copy(), v.copy()
    F, _ = _fe(x, box, per)
    out = []
    for _ in range(n_steps):
        oracle.kick(v, F, mass, 0.5 * dt)
        x = I.wrap(x + v * dt, box, per)
        F, E = _fe(x, box, per)
        oracle.kick(v, F, mass, 0.5 * dt)
        ke = 0.5 * (mass[:, None] * v * v).sum() * MVV
        out.append(ke + E.sum())
    return np.array(out)


def test_verlet_energy_error_is_second_order():
    x, box, per = _cell(3, 3, 3, disp=0.05, seed=2)
    rng = np.random.default_rng(5)
    mass = np.full(x.shape[0], I.CU_MASS_AMU)
    v = I.maxwell(x.shape[0], 600.0, I.CU_MASS_AMU, rng)
    e1 = _nve(2.0, 100, x, v, box, per, mass)
    e2 = _nve(1.0, 200, x, v, box, per, mass)
    _, E0 = _fe(x, box, per)
    tot0 = 0.5 * (mass[:, None] * v * v).sum() * MVV + E0.sum()
    err1 = np.max(np.abs(e1 - tot0))
    err2 = np.max(np.abs(e2 - tot0))
    assert err2 < 1e-3 * abs(tot0)
    assert 2.5 < err1 / err2 < 6.0, (err1, err2)


@pytest.mark.parametrize("mode", [0, 1])
def test_stopping_moves_energy_to_the_electrons(mode):
    n = 4
    mass = np.full(n, I.CU_MASS_AMU)
    rng = np.random.default_rng(3)
    v = rng.normal(0, 0.01, (n, 3))
    v[0] = [1.0, 0.5, -0.2]               # ~430 eV: above the cut
    K0 = 0.5 * mass * (v * v).sum(1) * MVV
    assert K0[0] > 10.0 and np.all(K0[1:] < 10.0)
    T = np.full(n, 500.0)
    A = np.array([0.3, -1e-4, 0.0, 2e-4])
    chi = np.ones(n, np.uint8)
    VC, beta, dt = 2.0e-6, 0.01, 0.5
    vv, TT, AA = v.copy(), T.copy(), A.copy()
    dKE, _ = oracle.couple(vv, mass, AA, TT, chi, mode=mode, frozen=0, seed=7, md_step=3, dt_md=dt,
                           gamma_fs=1e-3, VC=VC, stop_beta=beta, stop_ecut=10.0)
    K1 = 0.5 * mass * (vv * vv).sum(1) * MVV
    loss = K0[0] * (1.0 - math.exp(-2 * beta * dt))
    assert K1[0] == pytest.approx(K0[0] + A[0] - loss, rel=1e-12)
    assert (TT[0] - T[0]) * VC == pytest.approx(loss, rel=1e-9)
    assert np.array_equal(TT[1:], T[1:])
    # the same call without stopping: only the hand-over
    vv2, TT2, AA2 = v.copy(), T.copy(), A.copy()
    oracle.couple(vv2, mass, AA2, TT2, chi, mode=mode, frozen=0, seed=7, md_step=3, dt_md=dt,
                  gamma_fs=1e-3, VC=VC)
    assert np.array_equal(TT2, T)
    assert np.allclose(vv2[1:], vv[1:], rtol=0, atol=0)
