"""Distance-weighted pair rates (ehc_params.rate_shell_n) on the GPU against the
oracle's weighted substeps (oracle_pair_weights, oracle_substeps): the general
single-precision kernel and the FP64 kernel, conservation, and the windows'
plain fallback."""
import sys, os

import numpy as np
import pytest

from paper_1810_12357_gb300 import inputs as I

sys.path.insert(0, os.path.dirname(__file__))
from _drive import run_gpu, run_oracle   # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("flux_prec", [0, 1])
def test_weighted_rates_match_the_oracle(flux_prec):
    s = I.hot_spot_system(10, 8, peak=6000.0)
    p = dict(I.params_hotspot_fp64(), flux_prec=flux_prec, rate_shell_n=18, couple_mode=1, G=3e18, frozen=0)
    sim, _, _ = run_oracle(s, p, 3, 60)
    g, _, _ = run_gpu(s, p, 3, 60)
    Tg = g.get_te().cpu().numpy()
    err = float(np.max(np.abs(Tg - sim.T) / sim.T))
    # the single-precision path reads single-precision weights (r^2 rounded to float,
    # one rounded division); the FP64 path forms them as the oracle does,
    # S2 2^40 / (n_shell d2) in FP64, so it is held to the FP64 bar (the Langevin
    # normals are single precision on both paths, as in test_couple_parity)
    assert err < (1e-4 if flux_prec == 0 else 1e-11), err
    e = g.energy()
    assert abs(e["drift"]) < 1e-9
    # the weights change the result against uniform rates
    pu = dict(p, rate_shell_n=0)
    gu, _, _ = run_gpu(s, pu, 3, 60)
    du = float(np.max(np.abs(gu.get_te().cpu().numpy() - Tg) / Tg))
    assert du > 1e-4
    print(f"weighted rates flux_prec={flux_prec}: T_e err {err:.2e} vs oracle, {du:.2e} from uniform, "
          f"drift {e['drift']:.1e}")


def test_weighted_conservation_and_window_fallback():
    import torch
    from paper_1810_12357_gb300 import Ehc, EhcCheb
    s = I.track_system(8, 3, r0=6.0)
    p = dict(I.params_track(), G=0.0, rate_shell_n=18)
    a, _, _ = run_gpu(s, p, 1, 0)
    b, _, _ = run_gpu(s, p, 1, 0)
    T0 = a.get_te().cpu().numpy()
    w = EhcCheb(a, 16, 4, 0.05)
    fb, _ = w.step(1e30)
    b.substep(16)
    assert fb
    Ta = a.get_te().cpu().numpy()
    assert np.array_equal(Ta, b.get_te().cpu().numpy())
    assert abs(Ta.sum() - T0.sum()) < 1e-9 * T0.sum()
