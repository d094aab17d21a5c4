"""The bounds-checked build (libehc_checked.so, -DEHC_CHECKED: every gathered
neighbour and tile index is checked against its table, a violation sets an
error bit instead of reading out of bounds) runs the row-tile, general FP32
and FP64 substep paths without a violation and with results identical to the
normal library's."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(tmp_path, checked):
    out = str(tmp_path / ("checked.npz" if checked else "plain.npz"))
    env = dict(os.environ)
    env.pop("EHC_CHECKED", None)
    if checked:
        env["EHC_CHECKED"] = "1"
    r = subprocess.run([sys.executable, os.path.join(HERE, "_checked_run.py"), out], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(out)


def test_checked_build_matches_and_finds_no_violation(tmp_path):
    from paper_1810_12357_gb300 import build
    build.build(checked=True)
    a = _run(tmp_path, False)
    b = _run(tmp_path, True)
    for name in ("tiles", "general", "fp64"):
        assert int(b[name + "_err"][0]) == 0, name
        assert np.array_equal(a[name], b[name]), name
