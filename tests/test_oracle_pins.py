"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties an oracle function to a value that does not come from the
oracle itself: a brute-force search, a lattice count, a closed form, an
invariant of Eq. HeatTransport, the continuum limit of Eq. Kij, an energy
balance (Eqs. RateExchange, WorkDone, Xi), or published Philox vectors.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1810_12357_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- neighbours

@pytest.mark.parametrize("n,box,per,rc,seed", [
    (600, (14.0, 15.5, 16.0), (1, 1, 1), 4.0, 11),
    (900, (30.0, 12.0, 9.0), (1, 0, 1), 4.0, 12),
    (400, (8.5, 8.5, 25.0), (1, 1, 0), 3.3, 13),     # fewer than 3 cells per axis
    (1500, (20.0, 20.0, 20.0), (0, 0, 0), 5.0, 14),
])
def test_cell_search_equals_brute_force(n, box, per, rc, seed):
    s = I.random_box_system(n, box, seed, periodic=per)
    rb, cb = oracle.neighbors(s.x, s.box, s.periodic, rc, method="brute", cap_per_atom=200)
    rcl, ccl = oracle.neighbors(s.x, s.box, s.periodic, rc, method="cells", cap_per_atom=200)
    assert np.array_equal(rb, rcl)
    assert np.array_equal(cb, ccl)
    # symmetric list, no self pairs, distances within the cutoff
    rows = np.repeat(np.arange(n), np.diff(rb))
    assert not np.any(rows == cb)
    pairs = set(zip(rows.tolist(), cb.tolist()))
    assert all((j, i) in pairs for i, j in pairs)
    d = I.min_image(s.x[cb] - s.x[rows], s.box, s.periodic)
    assert np.sqrt((d * d).sum(1)).max() <= rc + 1e-5


@pytest.mark.parametrize("rc,count", [(3.0, 12), (4.0, 18), (5.0, 42)])
def test_perfect_fcc_shell_counts(rc, count):
    # FCC shells: 12 at a/sqrt2, 6 at a, 24 at a*sqrt(3/2) (= 4.427 A for Cu)
    a = I.CU_A
    x = I.fcc_lattice(5, 5, 5, a)
    box = np.array([5 * a] * 3)
    rp, col = oracle.neighbors(x, box, (1, 1, 1), rc, method="brute", cap_per_atom=64)
    assert np.all(np.diff(rp) == count)


def test_cutoff_is_inclusive_and_half_box_tie():
    # two atoms exactly r_c apart are neighbours; 1 grid unit further are not
    box = np.array([20.0, 20.0, 20.0])
    x = np.array([[1.0, 1.0, 1.0], [5.0, 1.0, 1.0], [1.0, 5.0 + 2.0 ** -20, 1.0]])
    rp, col = oracle.neighbors(x, box, (1, 1, 1), 4.0, method="brute")
    assert list(col[rp[0]:rp[1]]) == [1]
    # an atom exactly half a box away is counted once (minimum image)
    x2 = np.array([[0.0, 0.0, 0.0], [4.0, 0.0, 0.0]])
    rp2, col2 = oracle.neighbors(x2, np.array([8.0, 20.0, 20.0]), (1, 1, 1), 4.0, method="brute")
    assert list(np.diff(rp2)) == [1, 1]


# -------------------------------------------------------------- pair flux

def test_pair_flux_special_values():
    # f(a,b) = b(1-a)e^{a-b} - a(1-b)e^{b-a}  (Eq. HeatTransport, Delta e_ij = -(theta_i-theta_j))
    for b in (0.1, 0.37, 0.9):
        assert oracle.pair_flux(0.0, b) == pytest.approx(b * math.exp(-b), rel=1e-15)   # gain term only
        assert oracle.pair_flux(b, 0.0) == pytest.approx(-b * math.exp(-b), rel=1e-15)  # loss term only
        assert oracle.pair_flux(b, 1.0) == pytest.approx((1 - b) * math.exp(b - 1), rel=1e-15)
        assert oracle.pair_flux(1.0, b) == pytest.approx(-(1 - b) * math.exp(b - 1), rel=1e-15)


def test_pair_flux_antisymmetric_and_fixed_point():
    rng = np.random.default_rng(5)
    for a, b in rng.uniform(0, 1, size=(500, 2)):
        assert oracle.pair_flux(a, b) == -oracle.pair_flux(b, a)
        assert oracle.pair_flux(a, a) == 0.0


def test_pair_flux_linear_slope():
    # d f / d theta_j at theta_i = theta_j = t is 1 - 2 t (1 - t): heat runs from hot to cold
    for t in (0.015, 0.2, 0.5, 0.8):
        h = 1e-6
        slope = (oracle.pair_flux(t, t + h) - oracle.pair_flux(t, t - h)) / (2 * h)
        assert slope == pytest.approx(1 - 2 * t * (1 - t), rel=1e-8)


# ---------------------------------------------------------- substep invariants

def _sim(system, p):
    s = oracle.OracleSim(p, system.box, system.periodic, system.mass_amu, system.type,
                         depth=system.depth)
    s.set_te(system.Te)
    s.build(system.x, system.v)
    return s


def test_conservation_without_coupling():
    sysm = I.hot_spot_system(6, 1)
    p = I.params_hotspot_fp64()
    p["G"] = 0.0
    sim = _sim(sysm, p)
    s0 = sim.T.sum()
    sim.substeps(1000)
    assert abs(sim.T.sum() - s0) / s0 < 1e-13
    assert sim.T.max() < sysm.Te.max()  # the hot spot spreads
    e = sim.energy()
    assert abs(e["drift"]) < 1e-13


def test_uniform_fixed_point():
    sysm = I.hot_spot_system(4, 2)
    sysm.Te[:] = 1234.5
    p = I.params_hotspot_fp64()
    p["G"] = 0.0
    sim = _sim(sysm, p)
    sim.substeps(50)
    assert np.all(sim.T == 1234.5)
    # with coupling on and T_l == T_e the state stays put as well
    p["G"] = 1e17
    sim = _sim(sysm, p)
    sim.Tl[:] = 1234.5
    sim.substeps(50)
    assert np.all(sim.T == 1234.5)


def _decay_run(ncx, k_cells, n_sub, T0=300.0, amp=1.0, Tmax=2.0e4):
    a = I.CU_A
    x = I.fcc_lattice(ncx, 3, 3, a)
    box = np.array([ncx * a, 3 * a, 3 * a])
    k = 2 * math.pi / (k_cells * a)
    Te = T0 + amp * np.sin(k * x[:, 0])
    n = x.shape[0]
    sysm = I.System(x=x, v=np.zeros((n, 3)), Te=Te, box=box, periodic=np.array([1, 1, 1], np.int32),
                    mass_amu=np.array([I.CU_MASS_AMU]), type=np.zeros(n, np.int32), a=a)
    p = I.params_hotspot_fp64()
    p.update(G=0.0, Tmax=Tmax, kappa_mode=0)
    sim = _sim(sysm, p)
    basis = np.sin(k * x[:, 0])
    a0 = float((sim.T - T0) @ basis / (basis @ basis))
    sim.substeps(n_sub)
    a1 = float((sim.T - T0) @ basis / (basis @ basis))
    theta0 = T0 / Tmax
    c = 1 - 2 * theta0 * (1 - theta0)
    shell = I.fcc_shell_vectors(a, 4.0)
    lam = c * sim.K * float((1 - np.cos(k * shell[:, 0])).sum())
    return sim, p, a0, a1, lam, k, c


def test_fourier_decay_discrete_closed_form():
    # amplitude of a sin(k x) mode under forward Euler: (1 - dt lambda_k)^n
    sim, p, a0, a1, lam, k, c = _decay_run(10, 10, 400)
    pred = a0 * (1 - p["dt_sub"] * lam) ** 400
    assert a1 == pytest.approx(pred, rel=1e-6)
    assert a1 < 0.9 * a0


def test_fourier_decay_continuum_limit_of_eq_kij():
    # Eq. Kij makes the long-wavelength decay rate D k^2 c(theta), D = kappa_e / C_e
    sim, p, a0, a1, lam, k, c = _decay_run(40, 40, 2000)
    D = p["kappa0"] / sim.Ce * 1e20 * 1e-15          # m^2/s -> A^2/fs
    rate_meas = -math.log(a1 / a0) / (2000 * p["dt_sub"])
    assert rate_meas == pytest.approx(c * D * k * k, rel=5e-3)
    assert lam == pytest.approx(c * D * k * k, rel=5e-3)


# --------------------------------------------------------- coupling and ledger

@pytest.mark.parametrize("mode", [0, 1])
def test_exchange_balance(mode):
    sysm = I.hot_spot_system(4, 3, peak=8000.0)
    p = I.params_hotspot_fp64()
    p.update(frozen=0, couple_mode=mode, G=3e18)
    sim = _sim(sysm, p)
    v = sysm.v.copy()
    ke = lambda vv: float((0.5 * sim.mass * (vv * vv).sum(1) * oracle.MVV_EV).sum())
    ke0 = ke(v)
    lost = 0.0
    for step in range(5):
        if step:
            sim.build(sysm.x, v)
        sim.substeps(100)
        A = sim.A.copy()
        lost += float(A.sum())
        dKE = sim.couple(v, 1.0)
        chi = sim.chi.astype(bool)
        assert np.allclose(dKE[chi], A[chi], rtol=1e-9, atol=1e-18)
    assert sim.n_stopped == 0
    assert ke(v) - ke0 == pytest.approx(lost, rel=1e-10)
    assert abs(sim.energy()["drift"]) < 1e-12
    assert lost < 0 or lost > 0


def test_epsilon_guard_skips_both_sides():
    sysm = I.hot_spot_system(4, 4, peak=5000.0)
    sysm.v[7] = 0.0
    p = I.params_hotspot_fp64()
    p.update(frozen=0)
    sim = _sim(sysm, p)
    assert sim.chi[7] == 0 and sim.chi.sum() == sysm.n - 1
    sim.substeps(10)
    assert sim.A[7] == 0.0
    v = sysm.v.copy()
    sim.couple(v, 1.0)
    assert np.all(v[7] == 0.0)


def test_lattice_temperature_closed_forms():
    # two isolated atoms that see only each other: T = m |v1 - v2|^2 / (12 k_B)
    box = np.array([50.0, 50.0, 50.0])
    x = np.array([[10.0, 10.0, 10.0], [12.5, 10.0, 10.0]])
    v = np.array([[0.003, -0.001, 0.002], [-0.002, 0.0005, 0.001]])
    m = np.full(2, I.CU_MASS_AMU)
    rp, col = oracle.neighbors(x, box, (1, 1, 1), 4.0)
    Tl, Ks = oracle.lattice_temperature(rp, col, v, m)
    dv = v[0] - v[1]
    ref = I.CU_MASS_AMU * float(dv @ dv) * I.AMU_A2_FS2_EV / (12 * I.KB_EV)
    assert Tl[0] == pytest.approx(ref, rel=1e-13) and Tl[1] == pytest.approx(ref, rel=1e-13)
    assert Ks[0] == pytest.approx(0.5 * I.CU_MASS_AMU * float(v[0] @ v[0]) * I.AMU_A2_FS2_EV, rel=1e-14)
    # a common drift velocity is removed: T_l = 0
    x3 = I.fcc_lattice(3, 3, 3, I.CU_A)
    v3 = np.tile([0.01, -0.02, 0.005], (x3.shape[0], 1))
    rp3, col3 = oracle.neighbors(x3, np.array([3 * I.CU_A] * 3), (1, 1, 1), 4.0)
    Tl3, _ = oracle.lattice_temperature(rp3, col3, v3, np.full(x3.shape[0], I.CU_MASS_AMU))
    assert np.abs(Tl3).max() < 1e-9


def test_lattice_temperature_maxwell_mean():
    # Maxwell velocities at 300 K, N_j = 19: <T_l> = 300 (N_j - 1) / N_j, and 300 with dof_mode 1
    sysm = I.track_system(12, 9)
    rp, col = oracle.neighbors(sysm.x, sysm.box, sysm.periodic, 4.0)
    m = np.full(sysm.n, I.CU_MASS_AMU)
    Tl, _ = oracle.lattice_temperature(rp, col, sysm.v, m)
    Tl1, _ = oracle.lattice_temperature(rp, col, sysm.v, m, dof_mode=1)
    assert Tl.mean() == pytest.approx(300.0 * 18 / 19, rel=0.02)
    assert Tl1.mean() == pytest.approx(300.0, rel=0.02)


# ------------------------------------------------------------------ Philox

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]


def test_gauss3_statistics():
    g = np.array([oracle.gauss3(i, 7, 123) for i in range(20000)])
    assert abs(g.mean()) < 0.03 and g.std() == pytest.approx(1.0, abs=0.02)
    assert not np.array_equal(oracle.gauss3(1, 7, 123), oracle.gauss3(1, 8, 123))


def test_langevin_mode_moves_directions_not_energies():
    # Langevin hand-over: friction plus Philox random force, then the kinetic
    # energy of each atom is set to K_i + A_i, exactly as the damping
    # hand-over does; only the velocity directions differ.
    sysm = I.hot_spot_system(4, 6, peak=6000.0)
    out = {}
    for mode in (0, 1):
        p = I.params_hotspot_fp64()
        p.update(frozen=0, couple_mode=mode, G=1e19)
        sim = _sim(sysm, p)
        sim.substeps(200)
        v = sysm.v.copy()
        sim.couple(v, 1.0)
        out[mode] = (v, sim)
    v0, v1 = out[0][0], out[1][0]
    k0 = (v0 * v0).sum(1)
    k1 = (v1 * v1).sum(1)
    assert np.allclose(k0, k1, rtol=1e-12, atol=0)
    assert not np.allclose(v0, v1, rtol=1e-9, atol=0)
    # the random kick is small: sigma^2 ~ 2 g dt kB T_e / m per component
    sim = out[1][1]
    cosang = (v0 * v1).sum(1) / np.sqrt(k0 * k1)
    assert np.median(cosang) > 0.95


def test_langevin_stream_follows_the_atom_id():
    # The Langevin numbers of an atom are keyed by its id (default: its index):
    # ids equal to the indices change nothing; identical atoms labelled with
    # reversed ids come out reversed; two atoms with one id draw one set of
    # numbers; another MD step draws others.
    n = 64
    rng = np.random.default_rng(5)
    v1 = rng.normal(0.0, 0.03, 3)
    mass = np.full(n, 63.546)
    kw = dict(mode=1, frozen=0, seed=77, dt_md=0.1, gamma_fs=0.02, VC=2e-6)

    def run(ids, md_step=4, same=True):
        v = np.tile(v1, (n, 1)) if same else rng.normal(0.0, 0.03, (n, 3))
        A = np.full(n, 1e-4)
        T = np.full(n, 5000.0)
        chi = np.ones(n, dtype=np.uint8)
        dKE, _ = oracle.couple(v, mass, A, T, chi, md_step=md_step, rng_id=ids, **kw)
        return v, dKE

    v_def, d_def = run(None)
    v_idx, d_idx = run(np.arange(n))
    assert np.array_equal(v_def, v_idx) and np.array_equal(d_def, d_idx)
    v_rev, _ = run(np.arange(n)[::-1])
    assert np.array_equal(v_rev, v_def[::-1])
    assert not np.array_equal(v_rev, v_def)
    v_one, _ = run(np.full(n, 9))
    assert np.all(v_one == v_one[0]) and np.array_equal(v_one[0], v_def[9])
    v_step, _ = run(None, md_step=5)
    assert not np.any(np.all(v_step == v_def, axis=1))


# ------------------------------------------------------------- stability bound

def test_stability_bound_at_the_l_point():
    # FCC Cu at r_c = 4.0 A: 12 first and 6 second neighbours.  The mode
    # cos(pi (x + y + z) / a) (the L point) flips sign across all 6 second and
    # 6 of the 12 first neighbours, so its linearised rate is
    # lambda_L = K c(theta) sum_j (1 - cos k.r_j) = 24 K c(theta), the largest of
    # the lattice; forward Euler multiplies its amplitude by 1 - dt lambda_L per
    # substep, which stays bounded for dt lambda_L < 2 and grows above.
    a = I.CU_A
    x = I.fcc_lattice(4, 4, 4, a)
    n = x.shape[0]
    box = np.array([4 * a] * 3)
    per = np.array([1, 1, 1], dtype=np.int32)
    rowptr, col = oracle.neighbors(x, box, per, 4.0)
    assert np.all(np.diff(rowptr) == 18)
    mode = np.cos(np.pi * x.sum(axis=1) / a)
    assert np.allclose(np.abs(mode), 1.0) and abs(mode.sum()) < 1e-9
    shell = I.fcc_shell_vectors(a, 4.0)
    kvec = np.array([np.pi / a] * 3)
    assert float((1.0 - np.cos(shell @ kvec)).sum()) == pytest.approx(24.0, abs=1e-12)
    T0, amp, Tmax, K = 300.0, 1e-3, 1.0e5, 1.0
    th = T0 / Tmax
    lam = 24.0 * K * (1.0 - 2.0 * th * (1.0 - th))
    n_sub = 60
    for r in (0.95, 1.05):
        dt = r * 2.0 / lam
        T = T0 + amp * mode
        Tl = np.full(n, T0)
        chi = np.zeros(n, dtype=np.uint8)
        A = np.zeros(n)
        st, _ = oracle.substeps(rowptr, col, T, Tl, chi, A, n_sub, dt, Tmax, K, 0.0, 0.0)
        assert st == n_sub
        a1 = float((T - T0) @ mode / n)
        pred = amp * (1.0 - dt * lam) ** n_sub
        assert a1 == pytest.approx(pred, rel=1e-4)
        if r < 1:
            assert abs(a1) < 0.01 * amp
        else:
            assert abs(a1) > 100 * amp


# ------------------------------------------------------- Langevin statistics

def test_langevin_lattice_reaches_the_electron_temperature():
    # uniform T_e held fixed (a very large electronic heat capacity), strong
    # coupling, atoms at rest in space: the Langevin hand-over drives the lattice
    # to <KE> = (3/2) k_B T_e per atom (with the 3 (N_j - 1) degrees of freedom of
    # the centre-of-mass-free local temperature); statistical check at 3 sigma
    s = I.hot_spot_system(6, 5, peak=300.0)
    n = s.n
    Te = 900.0
    s.Te[:] = Te
    p = I.params_hotspot_fp64()
    p.update(frozen=0, couple_mode=1, G=3e18, gamma_Ce=1e12, dof_mode=1, dt_sub=1.0, Tmax=2.0e4)
    sim = _sim(s, p)
    v = s.v.copy()
    ke = lambda vv: 0.5 * sim.mass * (vv * vv).sum(1) * oracle.MVV_EV
    samples = []
    for step in range(600):
        if step:
            sim.build(s.x, v)
        sim.substeps(10)
        sim.couple(v, 10.0)
        if step >= 300:
            samples.append(float(ke(v).mean()))
    target = 1.5 * oracle.KB_EV * Te
    m = float(np.mean(samples))
    # per-atom kinetic energies are Gamma(3/2)-distributed: relative spread
    # sqrt(2/3) per atom; the 300 samples are correlated, count them as 5.
    # (3 N_j degrees of freedom would give 19/18 of the target, 5.6 % above,
    # outside this band.)
    sigma = target * math.sqrt(2.0 / 3.0) / math.sqrt(n * 5)
    assert abs(m - target) < 3.0 * sigma, (m, target, sigma)
    assert 19.0 / 18.0 * target - m > 3.0 * sigma
    assert abs(np.mean(sim.T) - Te) < 1e-3 * Te
