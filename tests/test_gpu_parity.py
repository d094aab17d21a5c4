"""CUDA path vs the CPU oracle, element by element, on the same seeded inputs.

Tolerances:
  neighbour lists            bit-exact (integer work)
  lattice temperature        1e-12 relative (FP64 on both sides, summation order differs)
  T_e, FP64 flux             1e-12 relative
  T_e, FP32 flux             1e-4 relative (the target for the single-precision pair flux)
  velocities after coupling  1e-10 relative (FP64; the Box-Muller log/cos/sin differ by ulps)
  energy drift               1e-9 relative (FP32 flux), 1e-12 (FP64 flux)
"""
import math

import numpy as np
import pytest

import oracle
from paper_1810_12357_gb300 import inputs as I

from _drive import run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def relerr(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


# ------------------------------------------------------------- neighbours

@pytest.mark.parametrize("case", ["hotspot", "random_periodic", "random_mixed", "few_cells", "track20"])
def test_neighbor_list_bit_exact(case):
    torch = _torch()
    from paper_1810_12357_gb300 import Ehc
    if case == "hotspot":
        s = I.hot_spot_system(10, 1)
        rc = 4.0
    elif case == "random_periodic":
        s = I.random_box_system(1500, (25.0, 31.0, 22.5), 21)   # ~23 neighbours on average
        rc = 4.0
    elif case == "random_mixed":
        s = I.random_box_system(800, (40.0, 18.0, 15.0), 22, periodic=(1, 0, 1))   # ~28 on average
        rc = 4.5
    elif case == "few_cells":
        s = I.random_box_system(700, (8.5, 9.0, 30.0), 23, periodic=(1, 1, 0))
        rc = 3.3
    else:
        s = I.track_system(20, 24, disp_sigma=0.1)
        rc = 4.0
    p = I.params_hotspot_fp64()
    p.update(rc=rc, max_neighbors=64)
    g = Ehc(p, s)
    g.set_te(s.Te)
    x = torch.as_tensor(s.x, device="cuda")
    v = torch.as_tensor(s.v, device="cuda")
    g.build_neighbors(x, v)
    rg, cg = g.export_neighbors()
    ro, co = oracle.neighbors(s.x, s.box, s.periodic, rc)
    assert np.array_equal(rg, ro)
    assert np.array_equal(cg, co)


def test_perfect_fcc_counts_on_gpu():
    torch = _torch()
    from paper_1810_12357_gb300 import Ehc
    s = I.track_system(12, 3)
    g = Ehc(I.params_track(), s)
    g.set_te(s.Te)
    g.build_neighbors(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.v, device="cuda"))
    rp, col = g.export_neighbors()
    assert np.all(np.diff(rp) == 18)
    assert g.energy()["max_count"] == 18


def test_lattice_temperature_parity():
    torch = _torch()
    from paper_1810_12357_gb300 import Ehc
    s = I.hot_spot_system(10, 1)
    s.v[5] = 0.0   # below the guard
    p = I.params_hotspot_fp64()
    g = Ehc(p, s)
    g.set_te(s.Te)
    g.build_neighbors(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.v, device="cuda"))
    Tl_g = g.get_lattice_temperature().cpu().numpy()
    rp, col = oracle.neighbors(s.x, s.box, s.periodic, p["rc"])
    Tl_o, Ks = oracle.lattice_temperature(rp, col, s.v, np.full(s.n, I.CU_MASS_AMU))
    chi = Ks >= p["eps_ke"]
    assert not chi[5] and Tl_g[5] == -1.0
    assert relerr(Tl_g[chi], Tl_o[chi]) < 1e-12


# ------------------------------------------------------------ substeps

def test_fp64_hotspot_1000_substeps():
    # 4,000-atom hot spot, frozen atoms, FP64 flux, 1,000 substeps of 1e-3 fs
    s = I.hot_spot_system(10, 1)
    p = I.params_hotspot_fp64()
    sim, _, _ = run_oracle(s, p, 1, 1000)
    g, _, _ = run_gpu(s, p, 1, 1000)
    Tg = g.get_te().cpu().numpy()
    assert relerr(Tg, sim.T) < 1e-12
    eg, eo = g.energy(), sim.energy()
    assert eg["E_e"] == pytest.approx(eo["E_e"], rel=1e-12)
    assert eg["E_lat"] == pytest.approx(eo["E_lat"], rel=1e-10)
    assert abs(eg["drift"]) < 1e-12


def test_fp32_track_10k_substeps():
    # track profile on 16^3 cells (16,384 atoms), FP32 flux, 100 MD steps x 100 substeps
    # (0.1 fs each), Langevin coupling, free flight: T_e within 1e-4, energy drift within 1e-9
    s = I.track_system(16, 2, r0=10.0)
    p = I.params_track()
    sim, xo, vo = run_oracle(s, p, 100, 100)
    g, xg, vg = run_gpu(s, p, 100, 100)
    Tg = g.get_te().cpu().numpy()
    err = relerr(Tg, sim.T)
    assert err < 1e-4, err
    eg = g.energy()
    assert abs(eg["drift"]) < 1e-9
    vg = vg.cpu().numpy()
    assert np.abs(vg - vo).max() / np.abs(vo).max() < 1e-6
    print(f"track16 FP32: max rel T_e err {err:.3e}, drift {eg['drift']:.3e}")


def test_fp32_matches_fp64_flux_single_step():
    s = I.hot_spot_system(8, 4, peak=6000.0)
    p64 = I.params_hotspot_fp64()
    p32 = dict(p64, flux_prec=0)
    g64, _, _ = run_gpu(s, p64, 1, 20)
    g32, _, _ = run_gpu(s, p32, 1, 20)
    assert relerr(g32.get_te().cpu().numpy(), g64.get_te().cpu().numpy()) < 1e-6


@pytest.mark.parametrize("mode", [0, 1])
def test_couple_parity(mode):
    s = I.hot_spot_system(6, 5, peak=9000.0)
    p = I.params_hotspot_fp64()
    p.update(frozen=0, couple_mode=mode, G=3e18)
    sim, xo, vo = run_oracle(s, p, 4, 100)
    g, xg, vg = run_gpu(s, p, 4, 100)
    assert relerr(g.get_te().cpu().numpy(), sim.T) < 1e-11
    vg = vg.cpu().numpy()
    assert np.abs(vg - vo).max() / np.abs(vo).max() < (1e-12 if mode == 0 else 1e-6)
    assert np.abs(xg.cpu().numpy() - xo).max() < 1e-9
    eg, eo = g.energy(), sim.energy()
    assert eg["E_lat"] == pytest.approx(eo["E_lat"], rel=1e-9)
    assert abs(eg["drift"]) < 1e-12


def test_philox_normals_match_oracle():
    # same Philox words and 24-bit uniforms on both sides; the GPU's Box-Muller
    # runs in single precision, the oracle's in double
    from paper_1810_12357_gb300 import philox_normals
    ids = np.concatenate([[0, 1, 2, 12345, 2 ** 33 + 7, 4_000_000 - 1], np.arange(1000, 3000)])
    out = philox_normals(ids, 17, 0xDEADBEEF12345).cpu().numpy()
    ref = np.array([oracle.gauss3(int(i), 17, 0xDEADBEEF12345) for i in ids])
    assert np.max(np.abs(out - ref) / np.maximum(1.0, np.abs(ref))) < 2e-6


def test_graph_replay_is_bitwise_equal():
    s = I.track_system(10, 6, r0=8.0)
    p1 = dict(I.params_track(), use_graph=1)
    p0 = dict(I.params_track(), use_graph=0)
    g1, _, v1 = run_gpu(s, p1, 3, 50)
    g0, _, v0 = run_gpu(s, p0, 3, 50)
    assert np.array_equal(g1.get_te().cpu().numpy(), g0.get_te().cpu().numpy())
    assert np.array_equal(v1.cpu().numpy(), v0.cpu().numpy())


def test_run_to_run_deterministic():
    s = I.track_system(10, 7, r0=8.0)
    p = I.params_track()
    a, _, va = run_gpu(s, p, 3, 40)
    b, _, vb = run_gpu(s, p, 3, 40)
    assert np.array_equal(a.get_te().cpu().numpy(), b.get_te().cpu().numpy())
    assert a.energy()["E_lat"] == b.energy()["E_lat"]


def test_odd_substep_counts_and_split_calls():
    # 37 + 63 substeps in two calls equal 100 in one call (mirror parity bookkeeping)
    torch = _torch()
    from paper_1810_12357_gb300 import Ehc
    s = I.track_system(8, 8, r0=6.0)
    p = I.params_track()
    res = []
    for split in ([100], [37, 63], [1, 2, 97]):
        g = Ehc(p, s)
        g.set_te(s.Te)
        x = torch.as_tensor(s.x, device="cuda")
        v = torch.as_tensor(s.v, device="cuda")
        g.build_neighbors(x, v)
        for k in split:
            g.substep(k)
        res.append(g.get_te().cpu().numpy())
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])


def test_checkpoint_resume_bit_identical(tmp_path):
    torch = _torch()
    from paper_1810_12357_gb300 import Ehc
    s = I.track_system(8, 9, r0=6.0)
    p = I.params_track()

    def steps(g, x, v, n):
        for _ in range(n):
            g.build_neighbors(x, v)
            g.substep(50)
            g.couple(v, 0.05)
            g.drift(x, v, 0.05)

    g = Ehc(p, s)
    g.set_te(s.Te)
    x = torch.as_tensor(s.x, device="cuda")
    v = torch.as_tensor(s.v, device="cuda")
    steps(g, x, v, 4)
    ref_T = g.get_te().cpu().numpy()
    ref_E = g.energy()

    g2 = Ehc(p, s)
    g2.set_te(s.Te)
    x2 = torch.as_tensor(s.x, device="cuda")
    v2 = torch.as_tensor(s.v, device="cuda")
    steps(g2, x2, v2, 2)
    path = str(tmp_path / "ck.bin")
    g2.save(path)
    g3 = Ehc(p, s)
    g3.load(path)
    steps(g3, x2, v2, 2)
    assert np.array_equal(g3.get_te().cpu().numpy(), ref_T)
    e3 = g3.energy()
    assert e3["E_lat"] == ref_E["E_lat"] and e3["E_e"] == pytest.approx(ref_E["E_e"], rel=1e-15)


def test_host_buffer_step_matches_device_calls():
    torch = _torch()
    from paper_1810_12357_gb300 import Ehc
    s = I.track_system(10, 10, r0=8.0)
    p = I.params_track()
    g, xg, vg = run_gpu(s, p, 2, 30)
    h = Ehc(p, s)
    h.set_te(s.Te)
    xh = torch.as_tensor(s.x).clone().pin_memory()
    vh = torch.as_tensor(s.v).clone().pin_memory()
    Te = torch.empty(s.n, dtype=torch.float64).pin_memory()
    for k in range(2):
        h.md_step_host(xh, vh, 30, k * 30 * p["dt_sub"], 30 * p["dt_sub"], Te)
    assert np.array_equal(Te.numpy(), g.get_te().cpu().numpy())
    assert np.array_equal(vh.numpy(), vg.cpu().numpy())
    assert np.array_equal(xh.numpy(), xg.cpu().numpy())


# ----------------------------------------------------------- error paths

def test_unstable_substep_refused():
    torch = _torch()
    from paper_1810_12357_gb300 import Ehc, EhcError
    s = I.hot_spot_system(10, 1)
    p = dict(I.params_hotspot_fp64(), dt_sub=0.01)   # the 0.01 fs step: dt * 36 K > 2
    g = Ehc(p, s)
    g.set_te(s.Te)
    g.build_neighbors(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.v, device="cuda"))
    assert g.energy()["stability"] > 2
    with pytest.raises(EhcError) as e:
        g.substep(10)
    assert e.value.code == -4


def test_range_error_is_sticky():
    torch = _torch()
    from paper_1810_12357_gb300 import Ehc, EhcError
    s = I.hot_spot_system(6, 1, peak=30000.0)
    p = dict(I.params_hotspot_fp64(), Tmax=2.0e4, flux_prec=0)
    g = Ehc(p, s)
    g.set_te(s.Te)
    g.build_neighbors(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.v, device="cuda"))
    g.substep(3)
    with pytest.raises(EhcError) as e:
        g.sync()
    assert e.value.code == -5


def test_neighbor_overflow_and_bounds_and_order():
    torch = _torch()
    from paper_1810_12357_gb300 import Ehc, EhcError
    s = I.hot_spot_system(6, 1)
    g = Ehc(dict(I.params_hotspot_fp64(), max_neighbors=12), s)
    with pytest.raises(EhcError) as e:
        g.build_neighbors(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.v, device="cuda"))
    assert e.value.code == -8     # no T_e yet
    g.set_te(s.Te)
    with pytest.raises(EhcError) as e:
        g.substep(1)
    assert e.value.code == -8     # no neighbour list yet
    with pytest.raises(EhcError) as e:
        g.build_neighbors(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.v, device="cuda"))
    assert e.value.code == -6
    s2 = I.random_box_system(200, (20.0, 20.0, 20.0), 3, periodic=(1, 1, 0))
    s2.x[3, 2] = 25.0
    g2 = Ehc(I.params_hotspot_fp64(), s2)
    g2.set_te(s2.Te)
    with pytest.raises(EhcError) as e:
        g2.build_neighbors(torch.as_tensor(s2.x, device="cuda"), torch.as_tensor(s2.v, device="cuda"))
    assert e.value.code == -9


def test_empty_and_tiny_systems():
    torch = _torch()
    from paper_1810_12357_gb300 import Ehc
    p = I.params_hotspot_fp64()
    g = Ehc(p, n=0, box=(20.0, 20.0, 20.0), periodic=(1, 1, 1), mass_amu=[I.CU_MASS_AMU], types=None)
    z = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    g.set_te(torch.zeros(0, dtype=torch.float64, device="cuda"))
    g.build_neighbors(z, z)
    g.substep(5)
    g.couple(z, 1.0)
    assert g.energy()["sum_T"] == 0.0
    # one isolated atom: no neighbours, coupling only
    s = I.random_box_system(1, (20.0, 20.0, 20.0), 4)
    sim, _, _ = run_oracle(s, p, 1, 50)
    gg, _, _ = run_gpu(s, p, 1, 50)
    assert relerr(gg.get_te().cpu().numpy(), sim.T) < 1e-13


def test_row_tile_path_matches_global_path():
    # W = 32 runs the shared-memory row-tile kernel, W = 64 the global-gather kernel
    s = I.track_system(12, 11, r0=8.0)
    p_tile = dict(I.params_track(), max_neighbors=32)
    p_glob = dict(I.params_track(), max_neighbors=64)
    a, _, va = run_gpu(s, p_tile, 3, 50)
    b, _, vb = run_gpu(s, p_glob, 3, 50)
    assert relerr(a.get_te().cpu().numpy(), b.get_te().cpu().numpy()) < 1e-7
    ea, eb = a.energy(), b.energy()
    assert abs(ea["drift"]) < 2e-9 and abs(eb["drift"]) < 2e-9


@pytest.mark.parametrize("flux_prec", [0, 1])
def test_laser_slab_source(flux_prec):
    # slab with free z surfaces and vacancies, Gaussian pulse absorbed below the top surface
    s = I.laser_slab_system(8, 20, 3)
    p = dict(I.params_laser(), flux_prec=flux_prec)
    sim, xo, vo = run_oracle(s, p, 4, 100, t0=45.0)
    g, xg, vg = run_gpu(s, p, 4, 100, t0=45.0)
    Tg = g.get_te().cpu().numpy()
    assert sim.T.max() > 1000.0       # the pulse heated the surface
    assert relerr(Tg, sim.T) < (1e-4 if flux_prec == 0 else 1e-11)
    eg, eo = g.energy(), sim.energy()
    assert eg["E_src"] == pytest.approx(eo["E_src"], rel=1e-6 if flux_prec == 0 else 1e-12)
    assert abs(eg["drift"]) < 1e-9
    assert abs(eo["drift"]) < 1e-12


def test_speed_outside_fixed_point_range_refused():
    # velocity components are summed exactly on a 2^-48 A/fs grid, which holds |v| < 256 A/fs
    torch = _torch()
    from paper_1810_12357_gb300 import Ehc, EhcError
    s = I.hot_spot_system(4, 2)
    s.v[7, 1] = -300.0
    g = Ehc(I.params_hotspot_fp64(), s)
    g.set_te(s.Te)
    with pytest.raises(EhcError) as e:
        g.build_neighbors(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.v, device="cuda"))
    assert e.value.code == -5


@pytest.mark.parametrize("T_lat", [300.0, 3000.0])
def test_skin_candidates_give_the_full_search_list(T_lat):
    """Neighbour lists taken from skin candidates (ehc_params.skin_A > 0: rebuilt only
    when an atom moved more than skin / 2) are the lists of the full cell search on
    the same cells (negative skin), in the same order: a track with free flight over
    12 MD steps (at 3,000 K the candidates are rebuilt along the way) gives bitwise
    the same temperatures and velocities, and its list equals the oracle's."""
    torch = _torch()
    s = I.track_system(12, 13, r0=8.0, disp_sigma=0.1, T_lat=T_lat)
    res = []
    for skin in (0.3, -0.3):
        p = dict(I.params_track(), skin=skin, dt_sub=5e-4)
        # MD steps of 0.5 fs: atoms move 0.2-0.6 A, past the skin's 0.15 A
        g, x, v = run_gpu(s, p, 12, 100, dt_md=0.5)
        res.append((g.get_te().cpu().numpy(), v.cpu().numpy(), x.cpu().numpy(), g))
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
    g = res[0][3]
    ro, co = oracle.neighbors(res[0][2], s.box, s.periodic, 4.0, cap_per_atom=32)
    # one more build on the final positions, against the oracle's list there
    g.build_neighbors(torch.as_tensor(res[0][2], device="cuda"), torch.as_tensor(res[0][1], device="cuda"))
    rg, cg = g.export_neighbors(cap_per_atom=32)
    assert np.array_equal(rg, ro) and np.array_equal(cg, co)
