"""Parity at the full size of the benchmark: the 4,000,000-atom swift-ion track
in the launch configuration bench.py times (row-tile kernel, graph replay).

* the neighbour list of all 4 M atoms equals the oracle's, bit for bit;
* after 10 substeps, sampled atoms equal the oracle run on their 10-hop
  neighbourhood (information travels one hop per substep, so the centre of a
  10-hop ball is exact after 10 substeps): T_e within 1e-4 relative;
* after a whole MD step (100 substeps, Langevin hand-over) the energy ledger
  closes to 1e-9;
and the same workload on 256,000 atoms over 100 MD steps (10,000 substeps)
against the oracle run of the whole sequence.
"""
import numpy as np
import pytest

import oracle
from paper_1810_12357_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N_SUB_SAMPLE = 10


def _ball(rowptr, col, seed, hops):
    """Atoms within `hops` neighbour hops of `seed`, and the neighbour list
    restricted to them (local ids; links leaving the ball are dropped, which
    only the outermost shell feels)."""
    n = rowptr.shape[0] - 1
    inball = np.zeros(n, dtype=bool)
    inball[seed] = True
    front = np.array([seed], dtype=np.int64)
    for _ in range(hops):
        cnt = rowptr[front + 1] - rowptr[front]
        idx = np.repeat(rowptr[front] - np.cumsum(cnt) + cnt, cnt) + np.arange(cnt.sum())
        nb = np.unique(col[idx])
        front = nb[~inball[nb]]
        inball[front] = True
    ball = np.flatnonzero(inball)
    loc = -np.ones(n, dtype=np.int64)
    loc[ball] = np.arange(ball.size)
    cnt = rowptr[ball + 1] - rowptr[ball]
    idx = np.repeat(rowptr[ball] - np.cumsum(cnt) + cnt, cnt) + np.arange(cnt.sum())
    lj = loc[col[idx]]
    li = np.repeat(np.arange(ball.size), cnt)
    keep = lj >= 0
    li, lj = li[keep], lj[keep]
    rp = np.zeros(ball.size + 1, dtype=np.int64)
    np.add.at(rp, li + 1, 1)
    return ball, loc, np.cumsum(rp), lj.astype(np.int32)


@pytest.fixture(scope="module")
def track():
    import torch
    from paper_1810_12357_gb300 import Ehc
    s = I.track_system(100, 2)
    p = I.params_track()
    g = Ehc(p, s)
    g.set_te(s.Te)
    x = torch.as_tensor(s.x, device="cuda")
    v = torch.as_tensor(s.v, device="cuda")
    g.build_neighbors(x, v)
    return s, p, g, x, v


def test_fullsize_neighbor_list_bit_exact(track):
    s, p, g, x, v = track
    rg, cg = g.export_neighbors(cap_per_atom=24)
    ro, co = oracle.neighbors(s.x, s.box, s.periodic, p["rc"], cap_per_atom=24)
    assert np.array_equal(rg, ro)
    assert np.array_equal(cg, co)


def test_fullsize_sampled_substeps(track):
    s, p, g, x, v = track
    g.substep(N_SUB_SAMPLE, 0.0)
    Tg = g.get_te().cpu().numpy()
    sim = oracle.OracleSim(p, s.box, s.periodic, s.mass_amu, s.type)
    sim.set_te(s.Te)
    sim.build(s.x, s.v)
    rng = np.random.default_rng(7)
    # samples across the track core, its flank and the far field
    rho = np.hypot(s.x[:, 0] - 0.5 * s.box[0], s.x[:, 1] - 0.5 * s.box[1])
    picks = np.concatenate([rng.choice(np.flatnonzero(rho < 8.0), 4, replace=False),
                            rng.choice(np.flatnonzero((rho > 15.0) & (rho < 40.0)), 4, replace=False),
                            rng.choice(np.flatnonzero(rho > 80.0), 4, replace=False)])
    worst = 0.0
    for a in picks:
        ball, loc, rp, col = _ball(sim.rowptr, sim.col, a, N_SUB_SAMPLE)
        T = s.Te[ball].copy()
        Tl = sim.Tl[ball].copy()
        chi = sim.chi[ball].copy()
        Aacc = np.zeros(ball.size)
        st, _ = oracle.substeps(rp, col, T, Tl, chi, Aacc, N_SUB_SAMPLE, p["dt_sub"], p["Tmax"], sim.K, sim.cG,
                                sim.VG)
        assert st == N_SUB_SAMPLE
        err = abs(Tg[a] - T[loc[a]]) / T[loc[a]]
        worst = max(worst, err)
    assert worst < 1e-4, worst
    print(f"full-size sampled T_e max rel err {worst:.3e}")


def test_fullsize_md_step_ledger(track):
    s, p, g, x, v = track
    g.substep(100 - N_SUB_SAMPLE, N_SUB_SAMPLE * p["dt_sub"])
    g.couple(v, 100 * p["dt_sub"])
    e = g.energy()
    assert abs(e["drift"]) < 1e-9
    assert e["n_stopped"] == 0


def test_256k_track_10k_substeps():
    # the track profile on 40^3 cells (256,000 atoms), FP32 flux, 100 MD steps x
    # 100 substeps of 1e-3 fs, Langevin coupling, free flight, against the oracle
    # run of the same sequence: T_e within 1e-4, ledger drift within 1e-9
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from _drive import run_gpu, run_oracle
    s = I.track_system(40, 2)
    p = I.params_track()
    sim, xo, vo = run_oracle(s, p, 100, 100)
    g, xg, vg = run_gpu(s, p, 100, 100)
    Tg = g.get_te().cpu().numpy()
    err = float(np.max(np.abs(Tg - sim.T) / sim.T))
    assert err < 1e-4, err
    e = g.energy()
    assert abs(e["drift"]) < 1e-9
    assert e["n_stopped"] == sim.n_stopped
    print(f"track40 (256k atoms) FP32, 10k substeps: max rel T_e err {err:.3e}, drift {e['drift']:.3e}")


def test_fullsize_local_form_sampled_substeps_and_ledger():
    """The LOCAL per-atom C_e / kappa_e form (ce_mode 1) in the launch configuration
    of `bench.py --ce-local` (4,000,000 atoms): sampled atoms after 10 substeps
    against oracle_substeps_local on their 10-hop neighbourhood (system T_lat of
    the build), then the ledger of a whole MD step."""
    import torch
    from paper_1810_12357_gb300 import Ehc
    s = I.track_system(100, 2)
    p = dict(I.params_track(), ce_mode=1)
    g = Ehc(p, s)
    g.set_te(s.Te)
    x = torch.as_tensor(s.x, device="cuda")
    v = torch.as_tensor(s.v, device="cuda")
    g.build_neighbors(x, v)
    g.substep(N_SUB_SAMPLE, 0.0)
    Tg = g.get_te().cpu().numpy()
    sim = oracle.OracleSim(p, s.box, s.periodic, s.mass_amu, s.type)
    sim.set_te(s.Te)
    sim.build(s.x, s.v)
    rng = np.random.default_rng(11)
    rho = np.hypot(s.x[:, 0] - 0.5 * s.box[0], s.x[:, 1] - 0.5 * s.box[1])
    picks = np.concatenate([rng.choice(np.flatnonzero(rho < 8.0), 4, replace=False),
                            rng.choice(np.flatnonzero((rho > 15.0) & (rho < 40.0)), 4, replace=False),
                            rng.choice(np.flatnonzero(rho > 80.0), 4, replace=False)])
    worst = 0.0
    for a in picks:
        ball, loc, rp, col = _ball(sim.rowptr, sim.col, a, N_SUB_SAMPLE)
        T = s.Te[ball].copy()
        Aacc = np.zeros(ball.size)
        st, _, _ = oracle.substeps_local(rp, col, T, sim.Tl[ball].copy(), sim.chi[ball].copy(), Aacc,
                                         N_SUB_SAMPLE, p["dt_sub"], p["Tmax"], kappa0=p["kappa0"],
                                         kappa_mode=p["kappa_mode"], Tlat=sim.Tlat, dim_d=p["dim_d"],
                                         S2_A2=p["zb2"], gamma=p["gamma_Ce"], cap_SI=sim.cap_SI(), G=p["G"],
                                         vatom_A3=sim.vatom)
        assert st == N_SUB_SAMPLE
        worst = max(worst, abs(Tg[a] - T[loc[a]]) / T[loc[a]])
    assert worst < 1e-4, worst
    g.substep(100 - N_SUB_SAMPLE, N_SUB_SAMPLE * p["dt_sub"])
    g.couple(v, 100 * p["dt_sub"])
    e = g.energy()
    assert abs(e["drift"]) < 1e-9
    print(f"full-size LOCAL form: sampled T_e max rel err {worst:.3e}, MD-step drift {e['drift']:.1e}")


def test_fullsize_forces():
    """Morse forces of all 4,000,000 atoms of the track (positions displaced by
    0.05 A so that the forces do not vanish by symmetry) against oracle_forces."""
    import torch
    from paper_1810_12357_gb300 import Ehc
    s = I.track_system(100, 2, disp_sigma=0.05)
    p = dict(I.params_track(), pot_D=0.3429, pot_alpha=1.3588, pot_r0=2.866)
    g = Ehc(p, s)
    g.set_te(s.Te)
    g.build_neighbors(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.v, device="cuda"))
    F, pe = g.forces()
    Fg = F.cpu().numpy()
    rowptr, col = oracle.neighbors(s.x, s.box, s.periodic, p["rc"], cap_per_atom=24)
    Fo, Eo = oracle.forces(s.x, s.box, s.periodic, rowptr, col, D=p["pot_D"], alpha=p["pot_alpha"],
                           r0=p["pot_r0"], rc=p["rc"])
    err = float(np.max(np.abs(Fg - Fo)))
    assert err < 2e-5, err
    assert pe == pytest.approx(float(Eo.sum()), rel=1e-6)
    print(f"full-size forces: max |dF| {err:.1e} eV/A of max {np.abs(Fo).max():.2f}, E_pot rel "
          f"{abs(pe - Eo.sum()) / abs(Eo.sum()):.1e}")


def test_fullsize_laser_slab():
    """The laser slab at its full size (60 x 60 x 200 cells, 2 % vacancies: 2,822,400
    atoms, free z surfaces): the neighbour list bit for bit, and after 10 substeps
    at the pulse peak, sampled atoms below the surface and deep in the slab against
    the oracle with the source term on their 10-hop neighbourhood."""
    import torch
    from paper_1810_12357_gb300 import Ehc
    s = I.laser_slab_system(60, 200, 3)
    p = I.params_laser()
    assert s.x.shape[0] == 2822400
    g = Ehc(p, s)
    g.set_te(s.Te)
    g.set_depth(s.depth)
    g.build_neighbors(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.v, device="cuda"))
    rg, cg = g.export_neighbors(cap_per_atom=24)
    sim = oracle.OracleSim(p, s.box, s.periodic, s.mass_amu, s.type, depth=s.depth)
    sim.set_te(s.Te)
    sim.build(s.x, s.v)
    assert np.array_equal(rg, sim.rowptr)
    assert np.array_equal(cg, sim.col)
    t0 = 45.0
    g.substep(N_SUB_SAMPLE, t0)
    Tg = g.get_te().cpu().numpy()
    rng = np.random.default_rng(5)
    picks = np.concatenate([rng.choice(np.flatnonzero(s.depth < 3.0), 4, replace=False),
                            rng.choice(np.flatnonzero((s.depth > 100.0) & (s.depth < 200.0)), 4, replace=False),
                            rng.choice(np.flatnonzero(s.depth > 600.0), 4, replace=False)])
    worst = 0.0
    for a in picks:
        ball, loc, rp, col = _ball(sim.rowptr, sim.col, a, N_SUB_SAMPLE)
        T = s.Te[ball].copy()
        Aacc = np.zeros(ball.size)
        st, _ = oracle.substeps(rp, col, T, sim.Tl[ball].copy(), sim.chi[ball].copy(), Aacc, N_SUB_SAMPLE,
                                p["dt_sub"], p["Tmax"], sim.K, sim.cG, sim.VG, depth=s.depth[ball].copy(),
                                source=p["laser"], Ce_SI=sim.Ce, vatom_A3=sim.vatom, t_start=t0)
        assert st == N_SUB_SAMPLE
        worst = max(worst, abs(Tg[a] - T[loc[a]]) / T[loc[a]])
    assert worst < 1e-4, worst
    # the source heated the surface layer within the 10 substeps
    assert Tg[s.depth < 3.0].mean() > s.Te[s.depth < 3.0].mean() + 1e-3
    print(f"full-size laser slab: list bit-exact, sampled T_e max rel err {worst:.3e}")


def test_fullsize_skin_lists_equal_the_oracle():
    """The bench's track configuration: lists from 0.3 A skin candidates on the
    4,000,000-atom track.  Four MD steps of 0.5 fs free flight (some thousand
    atoms cross a cell face in each, so atoms re-sort their candidate lists), then
    one more build: the list equals the oracle's on the final positions, and the
    temperatures equal those of the full search (negative skin: the same cells,
    searched in full every build) bit for bit."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    import torch
    from _drive import run_gpu
    s = I.track_system(100, 2)
    res = []
    for skin in (0.3, -0.3):
        p = dict(I.params_track(), skin=skin, dt_sub=5e-4)
        g, x, v = run_gpu(s, p, 4, 10, dt_md=0.5)
        res.append((g, x, v, g.get_te().cpu().numpy()))
    assert np.array_equal(res[0][3], res[1][3])
    g, x, v, _ = res[0]
    g.build_neighbors(x, v)
    rg, cg = g.export_neighbors(cap_per_atom=24)
    ro, co = oracle.neighbors(x.cpu().numpy(), s.box, s.periodic, 4.0, cap_per_atom=24)
    assert np.array_equal(rg, ro) and np.array_equal(cg, co)
