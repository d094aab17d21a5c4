"""The 4,000,000-atom swift-ion track over its full length against the FP64 oracle.

100 MD steps of 100 substeps (10,000 substeps of 1e-3 fs), Langevin hand-over,
free flight, neighbour rebuild every MD step, in the launch configuration
bench.py times (row-tile kernel, graph replay, lists from 0.3 A skin candidates:
the full search's lists).  The oracle's run of the same
sequence is cached by tests/_track4m_reference.py (about 8 minutes on 16 host
cores the first time).

* plain single-precision path: every atom's T_e within 1e-4 relative after MD
  steps 1, 10, 23, 50 and 100, ledger drift within 1e-9, the same number of
  stopped atoms;
* learned window (trained stage coefficients, 100-substep windows with the
  residual test and plain fallback): every atom's T_e within 1 % of the oracle
  after MD steps 23, 50 and 100, ledger drift within 1e-9.
"""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
import _track4m_reference as R  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ref():
    return R.load_or_compute(verbose=True)


def _max_rel(a, b):
    return float(np.max(np.abs(a - b) / b))


def test_track_4m_10k_substeps_plain(ref):
    import torch
    from paper_1810_12357_gb300 import Ehc
    s, p = R.workload()
    p = dict(p, skin=0.3)   # the bench's list path (the oracle searches in full)
    dt_md = R.N_SUB * p["dt_sub"]
    g = Ehc(p, s)
    g.set_te(s.Te)
    x = torch.as_tensor(s.x, device="cuda").contiguous()
    v = torch.as_tensor(s.v, device="cuda").contiguous()
    errs = {}
    for step in range(R.N_MD):
        g.build_neighbors(x, v)
        g.substep(R.N_SUB, step * dt_md)
        g.couple(v, dt_md)
        g.drift(x, v, dt_md)
        if step + 1 in R.SNAPSHOTS:
            errs[step + 1] = _max_rel(g.get_te().cpu().numpy(), ref[f"T_{step + 1}"])
    e = g.energy()
    print("4M track vs oracle, max rel T_e err after MD steps " +
          ", ".join(f"{k}: {v:.2e}" for k, v in errs.items()) +
          f"; drift {e['drift']:.2e} (oracle {float(ref['e_drift']):.1e}); v max abs diff "
          f"{float(np.max(np.abs(v.cpu().numpy() - ref['v']))):.1e} A/fs")
    assert max(errs.values()) < 1e-4, errs
    assert abs(e["drift"]) < 1e-9
    assert e["n_stopped"] == int(ref["n_stopped"])
    # the Langevin force's Box-Muller transform runs in single precision on the GPU
    assert float(np.max(np.abs(v.cpu().numpy() - ref["v"]))) < 1e-5 * float(np.abs(ref["v"]).max())


def test_track_4m_learned_window_against_oracle(ref):
    import torch
    from paper_1810_12357_gb300 import Ehc, EhcCheb, learned
    coeffs, info = learned.train_track_window()
    s, p = R.workload()
    p = dict(p, skin=0.3)   # the bench's list path (the oracle searches in full)
    dt_md = R.N_SUB * p["dt_sub"]
    n_w = 100
    g = Ehc(p, s)
    g.set_te(s.Te)
    x = torch.as_tensor(s.x, device="cuda").contiguous()
    v = torch.as_tensor(s.v, device="cuda").contiguous()
    w = None
    fallbacks = 0
    errs = {}
    for step in range(R.N_MD):
        g.build_neighbors(x, v)
        if w is None:
            w = EhcCheb(g, n_w, 15, 2.0 / 13.0, order=2)
            w.set_coefficients(*coeffs)
        fb, _ = w.step(100.0, step * dt_md)
        fallbacks += int(fb)
        g.couple(v, dt_md)
        g.drift(x, v, dt_md)
        if step + 1 in R.SNAPSHOTS:
            errs[step + 1] = _max_rel(g.get_te().cpu().numpy(), ref[f"T_{step + 1}"])
    e = g.energy()
    print("4M track, learned window vs oracle, max rel T_e err after MD steps " +
          ", ".join(f"{k}: {v:.2e}" for k, v in errs.items()) +
          f"; fallbacks {fallbacks} / {R.N_MD}; drift {e['drift']:.2e}; training {info['train_s']:.1f} s")
    assert max(errs[k] for k in (23, 50, 100)) < 1e-2, errs
    assert abs(e["drift"]) < 1e-9
