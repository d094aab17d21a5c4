"""Lattice side on the GPU against the oracle: shifted-force Morse forces and
energy (ehc_forces vs oracle_forces), a coupled velocity-Verlet run (kick, drift,
build, forces, kick, substeps, hand-over) step for step, the total energy
KE + PE + E_e of that run, the largest speed, and electronic stopping in the
hand-over (global and LOCAL forms)."""
import math

import numpy as np
import pytest

import oracle
from paper_1810_12357_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MORSE = dict(pot_D=0.3429, pot_alpha=1.3588, pot_r0=2.866)     # Cu, Girifalco and Weizer
MVV = 1.66053906660e-27 * 1.0e10 / 1.602176634e-19


def _params(**kw):
    # K = 2 d kappa0 / (C_e S2) = 5.3 / fs at kappa0 = 40: 100 substeps of 5e-3 fs per
    # 0.5 fs MD step stay below the stability limit (dt 2 n_max K = 0.95)
    p = dict(I.params_hotspot_fp64(), kappa0=40.0, dt_sub=5e-3, G=3e18, frozen=0, couple_mode=0, **MORSE)
    p.update(kw)
    return p


def _oracle_verlet(s, p, n_md, n_sub, dt_md):
    sim = oracle.OracleSim(p, s.box, s.periodic, s.mass_amu, s.type)
    sim.set_te(s.Te)
    x, v = s.x.copy(), s.v.copy()
    mass = sim.mass
    sim.build(x, v)
    F, _ = sim.forces()
    tot = []
    for step in range(n_md):
        oracle.kick(v, F, mass, 0.5 * dt_md)
        x = I.wrap(x + v * dt_md, s.box, s.periodic)
        sim.build(x, v)
        F, pe = sim.forces()
        oracle.kick(v, F, mass, 0.5 * dt_md)
        sim.substeps(n_sub, step * dt_md)
        sim.couple(v, dt_md)
        ke = 0.5 * float((mass[:, None] * v * v).sum()) * MVV
        tot.append(ke + pe + sim.energy()["E_e"])
    return sim, x, v, np.array(tot)


def _gpu_verlet(s, p, n_md, n_sub, dt_md):
    import torch
    from paper_1810_12357_gb300 import Ehc
    g = Ehc(p, s)
    g.set_te(s.Te)
    x = torch.as_tensor(s.x, device="cuda").contiguous()
    v = torch.as_tensor(s.v, device="cuda").contiguous()
    m = torch.as_tensor(s.mass_amu[s.type], device="cuda")
    g.build_neighbors(x, v)
    F, _ = g.forces()
    tot = []
    for step in range(n_md):
        g.kick(v, F, 0.5 * dt_md)
        g.drift(x, v, dt_md)
        g.build_neighbors(x, v)
        F, pe = g.forces(F)
        g.kick(v, F, 0.5 * dt_md)
        g.substep(n_sub, step * dt_md)
        g.couple(v, dt_md)
        ke = 0.5 * float((m[:, None] * v * v).sum()) * MVV
        tot.append(ke + pe + g.energy()["E_e"])
    torch.cuda.synchronize()
    return g, x.cpu().numpy(), v.cpu().numpy(), np.array(tot)


def test_forces_match_the_oracle():
    import torch
    from paper_1810_12357_gb300 import Ehc
    s = I.hot_spot_system(10, 8, disp_sigma=0.1)
    p = _params()
    g = Ehc(p, s)
    g.set_te(s.Te)
    g.build_neighbors(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.v, device="cuda"))
    F, pe = g.forces()
    Fg = F.cpu().numpy()
    rowptr, col = oracle.neighbors(s.x, s.box, s.periodic, p["rc"])
    Fo, Eo = oracle.forces(s.x, s.box, s.periodic, rowptr, col, D=p["pot_D"], alpha=p["pot_alpha"],
                           r0=p["pot_r0"], rc=p["rc"])
    # single-precision pair terms and sums: about 18 x 2^-24 of the largest pair force
    err = float(np.max(np.abs(Fg - Fo)))
    assert err < 2e-5, err
    assert np.abs(Fo).max() > 0.1
    assert pe == pytest.approx(float(Eo.sum()), rel=1e-6)
    print(f"Morse forces: max |F_gpu - F_oracle| {err:.1e} eV/A of max {np.abs(Fo).max():.2f}, "
          f"E_pot {pe:.6f} vs {Eo.sum():.6f} eV")


def test_verlet_run_matches_the_oracle_and_keeps_the_total_energy():
    s = I.hot_spot_system(10, 8, peak=6000.0, disp_sigma=0.05)
    p = _params()
    n_md, n_sub, dt_md = 12, 100, 0.5
    sim, xo, vo, to = _oracle_verlet(s, p, n_md, n_sub, dt_md)
    g, xg, vg, tg = _gpu_verlet(s, p, n_md, n_sub, dt_md)
    d = I.min_image(xg - xo, s.box, s.periodic)
    assert np.max(np.abs(d)) < 1e-6
    assert np.max(np.abs(vg - vo)) < 1e-5 * np.abs(vo).max()
    T = g.get_te().cpu().numpy()
    assert float(np.max(np.abs(T - sim.T) / sim.T)) < 1e-4
    # the electrons heated the lattice, and KE + PE + E_e stayed put up to the
    # Verlet error, on both sides alike
    assert sim.energy()["E_lat"] > 0.0
    ke0 = 0.5 * float((s.mass_amu[s.type][:, None] * s.v * s.v).sum()) * MVV
    assert np.max(np.abs(to - to[0])) < 2e-3 * ke0
    assert np.max(np.abs(tg - to)) < 1e-6 * abs(to[0])
    assert abs(g.energy()["drift"]) < 1e-9
    print(f"Verlet: total energy spread {np.ptp(to):.2e} eV (oracle) {np.ptp(tg):.2e} eV (GPU), "
          f"KE0 {ke0:.1f} eV, E_lat {sim.energy()['E_lat']:.3e} eV")


def test_max_speed():
    import torch
    from paper_1810_12357_gb300 import Ehc
    s = I.hot_spot_system(6, 2)
    s.v[17] = [0.7, -0.3, 0.2]
    g = Ehc(_params(), s)
    vmax = g.max_speed(torch.as_tensor(s.v, device="cuda"))
    assert vmax == pytest.approx(float(np.sqrt((s.v * s.v).sum(1)).max()), rel=1e-15)


@pytest.mark.parametrize("ce_mode,couple_mode", [(0, 0), (0, 1), (1, 0)])
def test_stopping_matches_the_oracle(ce_mode, couple_mode):
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from _drive import run_gpu, run_oracle
    s = I.hot_spot_system(8, 3, peak=3000.0)
    fast = np.array([5, 100, 900])
    # 28-37 eV atoms: above the 10 eV cut; each hands its electrons (2.5e-6 eV/K
    # per atom) about 1e-3 eV per MD step
    s.v[fast] = [[0.08, 0.05, -0.03], [-0.06, 0.07, 0.01], [0.02, 0.03, 0.1]]
    p = dict(I.params_hotspot_fp64(), frozen=0, couple_mode=couple_mode, ce_mode=ce_mode, G=3e18,
             stop_beta=1e-3, stop_ecut=10.0)
    sim, xo, vo = run_oracle(s, p, 2, 20)
    g, xg, vg = run_gpu(s, p, 2, 20)
    vg = vg.cpu().numpy()
    # the Langevin force's Box-Muller transform runs in single precision on the GPU
    assert np.max(np.abs(vg - vo)) < (1e-12 if couple_mode == 0 else 1e-6) * np.abs(vo).max()
    T = g.get_te().cpu().numpy()
    assert float(np.max(np.abs(T - sim.T) / sim.T)) < 1e-11
    # the stopped atoms' electrons took the energy
    sim0, _, _ = run_oracle(s, dict(p, stop_beta=0.0), 2, 20)
    assert np.all(sim.T[fast] > sim0.T[fast] + 1.0)
    eg, eo = g.energy(), sim.energy()
    assert eg["E_lat"] == pytest.approx(eo["E_lat"], rel=1e-10 if couple_mode == 0 else 1e-8)
    assert abs(eg["drift"]) < 1e-12 and abs(eo["drift"]) < 1e-12


def _cascade_system():
    s = I.hot_spot_system(10, 6, peak=300.0, disp_sigma=0.02)
    pka = 1234
    m = s.mass_amu[s.type[pka]]
    s.v[pka] = np.array([0.7071, 0.7071, 0.02]) * math.sqrt(2 * 1000.0 / (m * MVV))
    p = dict(I.params_track(), **MORSE, couple_mode=0, stop_beta=1e-5, stop_ecut=10.0)
    return s, p, pka


def _cascade_n_sub(vmax, dt_sub):
    # the step dt = min(0.1 fs, 0.02 A / max |v|) in whole electron substeps
    return max(1, int(round(min(0.1, 0.02 / vmax) / dt_sub)))


def _oracle_cascade(s, p, n_md):
    """The cascade on the oracle: velocity-Verlet with the oracle's forces and
    kicks, the largest speed from the FP64 velocities, substeps and hand-over."""
    sim = oracle.OracleSim(p, s.box, s.periodic, s.mass_amu, s.type)
    sim.set_te(s.Te)
    x, v = s.x.copy(), s.v.copy()
    mass = sim.mass
    sim.build(x, v)
    F, pe = sim.forces()
    tot0 = 0.5 * float((mass[:, None] * v * v).sum()) * MVV + pe + sim.energy()["E_e"]
    subs, tots = [], []
    t = 0.0
    for step in range(n_md):
        n_sub = _cascade_n_sub(float(np.sqrt((v * v).sum(axis=1)).max()), p["dt_sub"])
        dt = n_sub * p["dt_sub"]
        oracle.kick(v, F, mass, 0.5 * dt)
        x = I.wrap(x + v * dt, s.box, s.periodic)
        sim.build(x, v)
        F, pe = sim.forces()
        oracle.kick(v, F, mass, 0.5 * dt)
        sim.substeps(n_sub, t)
        sim.couple(v, dt)
        t += dt
        subs.append(n_sub)
        tots.append(0.5 * float((mass[:, None] * v * v).sum()) * MVV + pe + sim.energy()["E_e"])
    return sim, v, np.array(subs), tot0, np.array(tots)


def test_cascade_with_a_variable_step_matches_the_oracle():
    """A small cascade (Sec. 5 in miniature): a 1 keV knock-on atom aimed at a nearest
    neighbour in a 4,000-atom lattice, velocity-Verlet with the step
    dt = min(0.1 fs, 0.02 A / max |v|)
    (ehc_max_speed), the electron substeps of 1e-3 fs sized to each step,
    electronic stopping above 10 eV and the damping hand-over.  The oracle runs the
    same cascade: the GPU takes the same step sequence, its knock-on atom ends with
    the oracle's kinetic energy, and KE + PE + E_e stays within 0.3 eV on both."""
    import torch
    from paper_1810_12357_gb300 import Ehc
    s, p, pka = _cascade_system()
    m = s.mass_amu[s.type[pka]]
    n_md = 150
    sim, vo, subs_o, tot0_o, tots_o = _oracle_cascade(s, p, n_md)
    g = Ehc(p, s)
    g.set_te(s.Te)
    x = torch.as_tensor(s.x, device="cuda").contiguous()
    v = torch.as_tensor(s.v, device="cuda").contiguous()
    mm = torch.as_tensor(s.mass_amu[s.type], device="cuda")
    g.build_neighbors(x, v)
    F, pe = g.forces()
    e0 = g.energy()
    tot0 = 0.5 * float((mm[:, None] * v * v).sum()) * MVV + pe + e0["E_e"]
    ke_pka0 = 0.5 * m * float((v[pka] ** 2).sum()) * MVV
    subs, tots = [], []
    t = 0.0
    for step in range(n_md):
        n_sub = _cascade_n_sub(g.max_speed(v), p["dt_sub"])
        dt = n_sub * p["dt_sub"]
        g.kick(v, F, 0.5 * dt)
        g.drift(x, v, dt)
        g.build_neighbors(x, v)
        F, pe = g.forces(F)
        g.kick(v, F, 0.5 * dt)
        g.substep(n_sub, t)
        g.couple(v, dt)
        t += dt
        subs.append(n_sub)
        tots.append(0.5 * float((mm[:, None] * v * v).sum()) * MVV + pe + g.energy()["E_e"])
    subs, tots = np.array(subs), np.array(tots)
    ke_pka = 0.5 * m * float((v[pka] ** 2).sum()) * MVV
    ke_pka_o = 0.5 * m * float((vo[pka] ** 2).sum()) * MVV
    # the same variable step, MD step for MD step
    assert np.array_equal(subs, subs_o)
    assert subs.min() < 0.7 * subs.max()        # the step grew as the knock-on atom slowed
    # the knock-on atom gave up most of its energy, the same amount on both sides
    assert ke_pka < 0.5 * ke_pka0
    assert ke_pka == pytest.approx(ke_pka_o, rel=1e-3)
    assert float(np.max(np.abs(v.cpu().numpy() - vo))) < 1e-3 * float(np.abs(vo).max())
    # total energy KE + PE + E_e kept on both sides
    assert np.max(np.abs(tots - tot0)) < 0.3
    assert np.max(np.abs(tots_o - tot0_o)) < 0.3
    assert abs(g.energy()["drift"]) < 1e-9
    print(f"cascade: dt {p['dt_sub'] * subs.min():.3f}-{p['dt_sub'] * subs.max():.3f} fs over {t:.2f} fs, "
          f"knock-on KE {ke_pka0:.0f} -> {ke_pka:.2f} eV (oracle {ke_pka_o:.2f}), total energy spread "
          f"{np.ptp(tots):.2e} eV (oracle {np.ptp(tots_o):.2e})")
