"""Run a few MD steps of three configurations (row tiles, the general
single-precision kernel, FP64) and save the electronic temperatures and the
device error words to the .npz file named by argv[1].  Run once with the
normal library and once with EHC_CHECKED=1 (the bounds-checked build) by
tests/test_gpu_checked.py."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from _drive import run_gpu   # noqa: E402
from paper_1810_12357_gb300 import inputs as I   # noqa: E402


def cases():
    s = I.track_system(10, 4, r0=8.0)
    p = I.params_track()
    yield "tiles", s, p
    yield "general", s, dict(p, max_neighbors=64)
    h = I.hot_spot_system(8, 2, peak=5000.0)
    yield "fp64", h, dict(I.params_hotspot_fp64(), couple_mode=1, G=3e18, frozen=0)


def main(out):
    res = {}
    for name, s, p in cases():
        g, _, _ = run_gpu(s, p, 2, 30)
        res[name] = g.get_te().cpu().numpy()
        res[name + "_err"] = np.array([g.energy(check=False)["device_error"]])
    np.savez(out, **res)


if __name__ == "__main__":
    main(sys.argv[1])
