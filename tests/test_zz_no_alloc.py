"""The allocation-free energy entry point (collected last on purpose).

ehc_electron_energy_noalloc is for callers that cannot call cudaMalloc when they
need the electronic energy (an application with a fixed device memory pool, a
plugin that may not touch its host code's allocator, a loop that must not take
allocator locks).  It keeps its scratch in
a fixed device array inside the library.  Its results must agree with the
ledger that ehc_set_te / ehc_energy compute, on consecutive calls.
"""
import numpy as np
import pytest

from paper_1810_12357_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_energy_matches_ledger_twice():
    import torch
    from paper_1810_12357_gb300 import Ehc, EhcError, electron_energy_noalloc, load_library
    s = I.track_system(30, 5, r0=15.0)          # 108,000 atoms: 27 scratch blocks
    p = I.params_track()
    g = Ehc(p, s)
    g.set_te(s.Te)
    e = g.energy()
    vatom = float(np.prod(s.box)) / s.n
    Te = torch.as_tensor(s.Te, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for _ in range(2):
        electron_energy_noalloc(Te, p["gamma_Ce"], p["Ce_cap_kB"], vatom, out)
        torch.cuda.synchronize()
        sumT, maxT, E0 = out.cpu().numpy()
        assert sumT == pytest.approx(e["sum_T"], rel=1e-12)
        assert maxT == e["max_T"]
        assert E0 == pytest.approx(e["E_e0"], rel=1e-12)
    # a smaller input after a larger one reuses the scratch without stale partial sums
    Te2 = Te[:1000].clone()
    electron_energy_noalloc(Te2, p["gamma_Ce"], 0.0, vatom, out)
    torch.cuda.synchronize()
    ref = float((0.5 * p["gamma_Ce"] * s.Te[:1000] ** 2).sum() * vatom * 1e-30 / I.EV_J)
    assert out[2].item() == pytest.approx(ref, rel=1e-12)
    assert out[0].item() == pytest.approx(float(s.Te[:1000].sum()), rel=1e-13)
    # a NaN temperature is reported as the maximum, not dropped
    Te3 = Te[:5000].clone()
    Te3[1234] = float("nan")
    electron_energy_noalloc(Te3, p["gamma_Ce"], p["Ce_cap_kB"], vatom, out)
    torch.cuda.synchronize()
    assert np.isnan(out[1].item()) and np.isnan(out[0].item())
    # sizes beyond the fixed scratch are refused
    L = load_library()
    import ctypes
    code = L.ehc_electron_energy_noalloc(ctypes.c_void_p(Te.data_ptr()), 16_777_217, 96.6, 0.0, vatom,
                                         ctypes.c_void_p(out.data_ptr()), None)
    assert code == -1
