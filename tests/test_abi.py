"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every entry point include/ehc.h declares, and the
binding's structs match the C layout."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ehc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ehc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1810_12357_gb300 import build as B
    try:
        B.build()
    except RuntimeError as e:  # pragma: no cover - nvcc missing
        pytest.skip(f"cannot build libehc: {e}")
    import paper_1810_12357_gb300 as P
    return P.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    import paper_1810_12357_gb300 as P
    assert set(declared_functions()) == set(P._SIGS)


def test_struct_layout_matches_c():
    import paper_1810_12357_gb300 as P
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "ehc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(ehc_params), offsetof(ehc_params, seed),
         offsetof(ehc_params, use_graph), sizeof(ehc_energy_t), offsetof(ehc_energy_t, n_stopped),
         offsetof(ehc_energy_t, device_error));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    py = [ctypes.sizeof(P.ehc_params), P.ehc_params.seed.offset, P.ehc_params.use_graph.offset,
          ctypes.sizeof(P.ehc_energy_t), P.ehc_energy_t.n_stopped.offset, P.ehc_energy_t.device_error.offset]
    assert vals == py


def test_strerror_is_host_only(lib):
    # ehc_strerror touches no device state, so it can be called without a GPU
    for code in (0, -1, -4, -5, -9, -99):
        assert isinstance(lib.ehc_strerror(code), bytes)


def test_params_marshalling():
    import paper_1810_12357_gb300 as P
    from paper_1810_12357_gb300 import inputs as I
    q = P.make_params(I.params_laser())
    assert q.laser_on == 1 and q.couple_mode == 1 and q.kappa_mode == 1
    assert q.zb2_A2 == pytest.approx(12 * I.CU_A ** 2)
