"""Chebyshev window propagator (ehc_cheb_*) on the GPU against the FP64
reference oracle/window.py, plus its conservation, fallback and ledger."""
import numpy as np
import pytest

import oracle
from oracle import window as W
from paper_1810_12357_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _ctx(s, p):
    import torch
    from paper_1810_12357_gb300 import Ehc
    g = Ehc(p, s)
    g.set_te(s.Te)
    x = torch.as_tensor(s.x, device="cuda")
    v = torch.as_tensor(s.v, device="cuda")
    g.build_neighbors(x, v)
    return g, x, v


def test_coefficients_match_the_reference():
    from paper_1810_12357_gb300 import EhcCheb
    s = I.hot_spot_system(6, 1)
    g, _, _ = _ctx(s, dict(I.params_hotspot_fp64(), flux_prec=0))
    for st, eps in ((4, 0.05), (6, 0.3), (2, 0.0)):
        w = EhcCheb(g, 16, st, eps)
        nu, mut, kap, gam = w.coefficients()
        _, _, _, nu_o, mut_o = W.coefficients(st, eps)
        assert np.allclose(nu[1:], nu_o[1:], rtol=1e-13, atol=1e-15)
        assert np.allclose(mut[1:], mut_o[1:], rtol=1e-13, atol=1e-15)
        assert np.all(kap == 0.0) and np.all(gam == 0.0)
    for st in (4, 10):
        eps = 2.0 / 13.0
        w = EhcCheb(g, 16, st, eps, order=2)
        nu, mut, kap, gam = w.coefficients()
        _, _, mu_o, nu_o, mut_o, gam_o, _, _ = W.coefficients2(st, eps)
        assert np.allclose(nu[2:], nu_o[2:], rtol=1e-12, atol=1e-14)
        assert np.allclose(mut[1:], mut_o[1:], rtol=1e-12, atol=1e-14)
        assert np.allclose(kap[2:], 1.0 - mu_o[2:] - nu_o[2:], rtol=1e-10, atol=1e-13)
        assert np.allclose(gam[2:], gam_o[2:], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("peak,order", [(3000.0, 1), (12000.0, 1), (12000.0, 2)])
def test_one_window_matches_the_fp64_reference(peak, order):
    from paper_1810_12357_gb300 import EhcCheb
    s = I.hot_spot_system(10, 1, peak=peak)
    p = dict(I.params_hotspot_fp64(), flux_prec=0, G=0.0)
    g, _, _ = _ctx(s, p)
    K = g.energy()["K_per_fs"]
    st, eps = (4, 0.05) if order == 1 else (6, 2.0 / 13.0)
    w = EhcCheb(g, 16, st, eps, order=order)
    fb, rho = w.step(1e30)
    assert not fb
    Tg = g.get_te().cpu().numpy()
    rowptr, col = oracle.neighbors(s.x, s.box, s.periodic, p["rc"])
    win = W.window if order == 1 else W.window2
    y, _ = win(rowptr, col, s.Te / p["Tmax"], K, 16 * p["dt_sub"], st, eps)
    To = y * p["Tmax"]
    assert np.max(np.abs(Tg - To) / To) < 1e-5
    assert np.max(np.abs(To - s.Te)) > 1.0        # the window did move the temperatures
    # every stage keeps the sum of temperatures
    assert abs(Tg.sum() - s.Te.sum()) < 1e-6 * s.Te.sum()


def test_fallback_is_the_plain_path():
    # tau = 0: the window is redone with plain substeps, bit for bit
    import torch
    from paper_1810_12357_gb300 import Ehc, EhcCheb
    s = I.track_system(8, 22, r0=6.0)
    p = I.params_track()
    a, x, v = _ctx(s, p)
    b, _, _ = _ctx(s, p)
    w = EhcCheb(a, 16, 4, 0.05)
    for _ in range(3):
        fb, rho = w.step(0.0)
        assert fb and rho > 0.0
        b.substep(16)
    assert np.array_equal(a.get_te().cpu().numpy(), b.get_te().cpu().numpy())
    assert w.stats() == (3, 3)


def test_accepted_windows_keep_the_ledger_closed():
    from paper_1810_12357_gb300 import EhcCheb
    s = I.hot_spot_system(8, 3, peak=6000.0)
    p = dict(I.params_hotspot_fp64(), flux_prec=0, frozen=0, couple_mode=1, G=3e18)
    g, x, v = _ctx(s, p)
    w = EhcCheb(g, 16, 4, 0.05)
    for step in range(3):
        if step:
            g.build_neighbors(x, v)
        for _ in range(4):
            fb, _ = w.step(1e30)
            assert not fb
        g.couple(v, 64 * p["dt_sub"])
    e = g.energy()
    assert abs(e["drift"]) < 1e-8
    assert e["E_lat"] != 0.0


def test_window_run_matches_the_reference_run():
    # 20 windows of 25 substeps (5 stages) on a 55,296-atom track profile,
    # coupling off: the GPU windows follow the FP64 reference windows; both
    # differ from the plain substeps by about a per cent while the initial
    # front is sharp (see the one-window bounds of the reference)
    import torch
    from paper_1810_12357_gb300 import EhcCheb
    s = I.track_system(24, 2, r0=20.0)
    p = dict(I.params_track(), G=0.0)
    g, _, _ = _ctx(s, p)
    K = g.energy()["K_per_fs"]
    w = EhcCheb(g, 25, 5, 0.05)
    for _ in range(20):
        fb, _ = w.step(1e30)
        assert not fb
    Tg = g.get_te().cpu().numpy()
    sim = oracle.OracleSim(p, s.box, s.periodic, s.mass_amu, s.type)
    sim.set_te(s.Te)
    sim.build(s.x, s.v)
    th = s.Te / p["Tmax"]
    for _ in range(20):
        th, _ = W.window(sim.rowptr, sim.col, th, K, 25 * p["dt_sub"], 5, 0.05)
    To = th * p["Tmax"]
    sim.substeps(500)
    err_ref = float(np.max(np.abs(Tg - To) / To))
    err_plain = float(np.max(np.abs(Tg - sim.T) / sim.T))
    print(f"window run: vs FP64 windows {err_ref:.2e}, vs plain substeps {err_plain:.2e}")
    assert err_ref < 1e-5
    assert err_plain < 3e-2
