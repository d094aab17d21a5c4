"""Failure detection on the GPU without a fault: the bounded mbarrier wait of the
row-tile kernels run out on purpose (a phase that nothing completes) returns
EHC_E_TIMEOUT to the host within its poll budget, the same wait on a phase that
completes returns EHC_OK, and the context keeps working afterwards."""
import os
import sys
import time

import numpy as np
import pytest

from paper_1810_12357_gb300 import inputs as I

sys.path.insert(0, os.path.dirname(__file__))
from _drive import run_gpu   # noqa: E402

pytestmark = pytest.mark.gpu

EHC_E_TIMEOUT = -7


def test_bounded_wait_reports_a_timeout_and_the_context_stays_usable():
    s = I.hot_spot_system(6, 2)
    p = I.params_hotspot_fp64()
    g, _, _ = run_gpu(s, p, 1, 10)
    T0 = g.get_te().cpu().numpy()
    assert g.probe_wait(1000, complete=True) == 0
    t = time.perf_counter()
    assert g.probe_wait(1000, complete=False) == EHC_E_TIMEOUT
    assert time.perf_counter() - t < 5.0
    # a larger budget runs out as well, and nothing else was touched
    assert g.probe_wait(100000, complete=False) == EHC_E_TIMEOUT
    g.substep(10)
    e = g.energy()
    assert e["device_error"] == 0
    assert np.all(np.isfinite(g.get_te().cpu().numpy()))
    assert not np.array_equal(g.get_te().cpu().numpy(), T0)
