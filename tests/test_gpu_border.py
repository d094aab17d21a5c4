"""Fixed-temperature electron border (ehc_set_border) on the GPU against the
oracle's border (oracle/ehc_oracle.c: oracle_substeps with Tfix): every path
(row tiles in FP32, the general FP32 kernel, FP64), the reservoir in the
ledger, and the border switched on and off between builds."""
import sys, os

import numpy as np
import pytest

import oracle
from paper_1810_12357_gb300 import inputs as I

sys.path.insert(0, os.path.dirname(__file__))
from _drive import run_gpu, run_oracle   # noqa: E402

pytestmark = pytest.mark.gpu


def _shell(s, width):
    # atoms within `width` A of a box face
    edge = np.any((s.x < width) | (s.x > s.box - width), axis=1)
    return edge, np.where(edge, 300.0, np.nan)


@pytest.mark.parametrize("flux_prec,use_graph", [(0, 1), (0, 0), (1, 1)])
def test_border_matches_the_oracle(flux_prec, use_graph):
    s = I.hot_spot_system(10, 5, peak=6000.0)
    p = dict(I.params_hotspot_fp64(), flux_prec=flux_prec, use_graph=use_graph, couple_mode=1, G=3e18,
             frozen=0)
    edge, Tfix = _shell(s, 4.0)
    s.Te[edge] = 300.0
    sim, _, _ = run_oracle(s, p, 4, 50, border=Tfix)
    g, _, _ = run_gpu(s, p, 4, 50, border=Tfix)
    Tg = g.get_te().cpu().numpy()
    err = float(np.max(np.abs(Tg - sim.T) / sim.T))
    tol = 1e-4 if flux_prec == 0 else 1e-12
    assert err < tol, err
    assert np.max(np.abs(Tg[edge] - 300.0)) < 1e-9
    e, eo = g.energy(), sim.energy()
    assert e["E_res"] == pytest.approx(eo["E_res"], rel=1e-4 if flux_prec == 0 else 1e-10)
    assert e["E_res"] > 0.0
    assert abs(e["drift"]) < 1e-9
    print(f"border flux_prec={flux_prec} graph={use_graph}: T_e err {err:.2e}, E_res {e['E_res']:.4e} eV "
          f"(oracle {eo['E_res']:.4e}), drift {e['drift']:.1e}")


def test_general_fp32_kernel_with_border():
    # a neighbour table wider than 32 takes the general single-precision kernel
    s = I.hot_spot_system(8, 6, peak=3000.0)
    p = dict(I.params_hotspot_fp64(), flux_prec=0, G=0.0, max_neighbors=64)
    edge, Tfix = _shell(s, 4.0)
    s.Te[edge] = 300.0
    sim, _, _ = run_oracle(s, p, 2, 40, border=Tfix)
    g, _, _ = run_gpu(s, p, 2, 40, border=Tfix)
    Tg = g.get_te().cpu().numpy()
    assert np.max(np.abs(Tg - sim.T) / sim.T) < 1e-4
    assert abs(g.energy()["drift"]) < 1e-9


def test_empty_border_and_switching():
    import torch
    from paper_1810_12357_gb300 import Ehc
    s = I.hot_spot_system(8, 7, peak=5000.0)
    p = dict(I.params_hotspot_fp64(), flux_prec=0, G=0.0)
    # all NaN: bitwise the plain method
    g0, _, _ = run_gpu(s, p, 2, 30)
    g1, _, _ = run_gpu(s, p, 2, 30, border=np.full(s.n, np.nan))
    assert np.array_equal(g0.get_te().cpu().numpy(), g1.get_te().cpu().numpy())
    assert g1.energy()["E_res"] == 0.0
    # on for one MD step, off for the next: the ledger keeps the reservoir of the first
    edge, Tfix = _shell(s, 4.0)
    Te = s.Te.copy()
    Te[edge] = 300.0
    g = Ehc(p, s)
    g.set_te(Te)
    x = torch.as_tensor(s.x, device="cuda")
    v = torch.as_tensor(s.v, device="cuda")
    g.set_border(Tfix)
    g.build_neighbors(x, v)
    g.substep(40)
    e1 = g.energy()
    g.set_border(None)
    g.build_neighbors(x, v)
    g.substep(40)
    e2 = g.energy()
    assert e1["E_res"] > 0.0 and e2["E_res"] == pytest.approx(e1["E_res"], rel=1e-12)
    assert abs(e2["drift"]) < 1e-9
    Tg = g.get_te().cpu().numpy()
    assert np.max(Tg[edge]) > 300.0 + 1e-6    # free again: the shell warms


def test_window_propagator_falls_back_with_a_border():
    import torch
    from paper_1810_12357_gb300 import Ehc, EhcCheb
    s = I.track_system(8, 22, r0=6.0)
    p = I.params_track()
    edge, Tfix = _shell(s, 3.0)
    s.Te[edge] = 300.0
    a, _, _ = run_gpu(s, p, 1, 0, border=Tfix)
    b, _, _ = run_gpu(s, p, 1, 0, border=Tfix)
    w = EhcCheb(a, 16, 4, 0.05)
    fb, _ = w.step(1e30)
    b.substep(16)
    assert fb
    assert np.array_equal(a.get_te().cpu().numpy(), b.get_te().cpu().numpy())
