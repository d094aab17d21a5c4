"""LOCAL per-atom C_e / kappa_e form (ehc_params.ce_mode = 1) on the GPU against the
oracle's oracle_substeps_local: the general single-precision kernel (energy state
as a float pair, mirror rebuilt from it) and the FP64 kernel, with Langevin and
damping hand-over, the C_e cap, distance weights and the laser source; the
ledger's E_e = sum_i V_atom U(T_i); and the paths that refuse the form or
advance it with plain substeps."""
import os
import sys

import numpy as np
import pytest

from paper_1810_12357_gb300 import inputs as I

sys.path.insert(0, os.path.dirname(__file__))
from _drive import run_gpu, run_oracle   # noqa: E402

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.mark.parametrize("flux_prec,kappa_mode,couple_mode", [(0, 1, 1), (0, 0, 0), (1, 1, 1), (1, 0, 0)])
def test_local_form_matches_the_oracle(flux_prec, kappa_mode, couple_mode):
    s = I.hot_spot_system(10, 8, peak=6000.0)
    p = dict(I.params_hotspot_fp64(), flux_prec=flux_prec, ce_mode=1, kappa_mode=kappa_mode,
             couple_mode=couple_mode, G=3e18, frozen=0)
    sim, _, _ = run_oracle(s, p, 3, 60)
    g, _, _ = run_gpu(s, p, 3, 60)
    Tg = g.get_te().cpu().numpy()
    err = relerr(Tg, sim.T)
    # FP32 pair terms: 1e-4 of T (the bar of the global form); FP64: rounding order only
    assert err < (1e-4 if flux_prec == 0 else 1e-11), err
    eg, eo = g.energy(), sim.energy()
    assert eg["E_e"] == pytest.approx(eo["E_e"], rel=1e-6 if flux_prec == 0 else 1e-12)
    assert eg["E_lat"] == pytest.approx(eo["E_lat"], rel=1e-5 if flux_prec == 0 else 1e-10)
    assert abs(eg["drift"]) < 1e-9
    assert abs(eo["drift"]) < 1e-12
    # the local form is not the global one on this profile
    gg, _, _ = run_gpu(s, dict(p, ce_mode=0), 3, 60)
    d = relerr(gg.get_te().cpu().numpy(), Tg)
    assert d > 1e-3
    print(f"local form flux_prec={flux_prec} kappa_mode={kappa_mode}: T_e err {err:.2e}, "
          f"drift {eg['drift']:.1e}, {d:.2e} from the global form")


def test_local_form_across_the_cap_with_weights():
    # a 60,000 K spot on 20,000 K: the capped atoms' C_e is 3 k_B per atom
    s = I.hot_spot_system(10, 5, T0=20000.0, peak=60000.0)
    p = dict(I.params_track(), ce_mode=1, rate_shell_n=18, dt_sub=2e-4)
    sim, _, _ = run_oracle(s, p, 3, 50)
    g, _, _ = run_gpu(s, p, 3, 50)
    Tc = 3.0 * 1.380649e-23 / (I.CU_A ** 3 / 4.0 * 1e-30) / p["gamma_Ce"]
    assert s.Te.max() > Tc > s.Te.min()
    Tg = g.get_te().cpu().numpy()
    assert relerr(Tg, sim.T) < 1e-4
    eg, eo = g.energy(), sim.energy()
    assert eg["E_e"] == pytest.approx(eo["E_e"], rel=1e-6)
    assert abs(eg["drift"]) < 1e-9


@pytest.mark.parametrize("flux_prec", [0, 1])
def test_local_form_with_the_laser_source(flux_prec):
    s = I.laser_slab_system(8, 20, 3)
    p = dict(I.params_laser(), flux_prec=flux_prec, ce_mode=1)
    sim, _, _ = run_oracle(s, p, 4, 100, t0=45.0)
    g, _, _ = run_gpu(s, p, 4, 100, t0=45.0)
    Tg = g.get_te().cpu().numpy()
    assert sim.T.max() > 1000.0
    assert relerr(Tg, sim.T) < (1e-4 if flux_prec == 0 else 1e-11)
    eg, eo = g.energy(), sim.energy()
    assert eg["E_src"] == pytest.approx(eo["E_src"], rel=1e-6 if flux_prec == 0 else 1e-12)
    assert abs(eg["drift"]) < 1e-9
    assert abs(eo["drift"]) < 1e-12


def test_local_track_ledger_and_parity():
    """The track's profile (20,000 K core on 300 K, Langevin, cap) at 32,000 atoms,
    3 MD steps of 40 substeps, while the core still spreads (the electrons of this
    cell equilibrate within about 0.6 fs): T_e against the oracle and the ledger's
    drift."""
    s = I.track_system(20, 7, peak=20000.0, r0=8.0)
    p = dict(I.params_track(), ce_mode=1)
    sim, _, _ = run_oracle(s, p, 3, 40)
    assert sim.T.max() > 3.0 * sim.T.min()
    g, _, _ = run_gpu(s, p, 3, 40)
    Tg = g.get_te().cpu().numpy()
    err = relerr(Tg, sim.T)
    assert err < 1e-4, err
    e = g.energy()
    assert e["stability"] < 2.0
    assert abs(e["drift"]) < 1e-9
    print(f"local track: T_e err {err:.2e}, drift {e['drift']:.1e}, stability {e['stability']:.3f}")


def test_local_form_refusals_and_plain_fallbacks():
    import torch
    from paper_1810_12357_gb300 import Ehc, EhcBatch, EhcCheb, EhcError, EhcNN
    s = I.track_system(8, 3, r0=6.0)
    p = dict(I.params_track(), ce_mode=1, G=0.0)
    a, _, _ = run_gpu(s, p, 1, 0)
    b, _, _ = run_gpu(s, p, 1, 0)
    with pytest.raises(EhcError) as e:
        a.set_border(np.full(s.x.shape[0], 300.0))
    assert e.value.code == -8
    # the window advances a LOCAL context with plain substeps
    w = EhcCheb(a, 16, 4, 0.05)
    fb, _ = w.step(1e30)
    b.substep(16)
    assert fb
    assert np.array_equal(a.get_te().cpu().numpy(), b.get_te().cpu().numpy())
    with pytest.raises(EhcError):
        EhcNN(a)
    with pytest.raises(EhcError):
        EhcBatch(p, [s, s])


def test_local_row_tiles_equal_the_general_kernel():
    """The LOCAL form on the row tiles (16-bit tile indices, the default for FCC
    lists) and on the general kernel (forced by a table wider than 32 slots): the
    same pair terms in the same order with the same series order per substep,
    TwoSum sums, the same update."""
    s = I.track_system(16, 5, peak=20000.0, r0=8.0)
    p = dict(I.params_track(), ce_mode=1)
    a, _, _ = run_gpu(s, p, 3, 40)
    b, _, _ = run_gpu(s, dict(p, max_neighbors=40), 3, 40)
    Ta, Tb = a.get_te().cpu().numpy(), b.get_te().cpu().numpy()
    d = relerr(Ta, Tb)
    assert d < 1e-7, d
    assert abs(a.energy()["drift"]) < 1e-12
    print(f"LOCAL row tiles vs general kernel: {d:.1e}")
