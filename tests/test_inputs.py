"""The seeded input generators against the workloads they stand for (sizes,
temperature profiles, surfaces and vacancies, replica sizes) and their
reproducibility.  Both the oracle and the CUDA path read these inputs, so a
wrong recipe would pass every parity test; these checks tie it to the stated
configurations.  CPU only."""
import math

import numpy as np
import pytest

from paper_1810_12357_gb300 import inputs as I

A = I.CU_A


def _kinetic_temperature(s):
    m = s.mass_amu[0] * I.AMU_A2_FS2_EV
    ke = 0.5 * m * (s.v * s.v).sum(axis=1)
    return 2.0 * ke.mean() / (3.0 * I.KB_EV)


def test_fcc_lattice_counts_and_spacing():
    x = I.fcc_lattice(3, 4, 5, A)
    assert x.shape == (4 * 3 * 4 * 5, 3)
    # nearest neighbours at a / sqrt(2), 12 of them, inside the periodic box
    box = np.array([3 * A, 4 * A, 5 * A])
    d = I.min_image(x[1:] - x[0], box, np.array([1, 1, 1]))
    r = np.sqrt((d * d).sum(axis=1))
    assert np.isclose(r.min(), A / math.sqrt(2.0), rtol=1e-12)
    assert int(np.sum(np.isclose(r, A / math.sqrt(2.0), rtol=1e-9))) == 12


def test_hot_spot_system_is_the_4000_atom_configuration():
    s = I.hot_spot_system(10, 1)
    assert s.n == 4000 and np.allclose(s.box, 10 * A) and list(s.periodic) == [1, 1, 1]
    # Gaussian displacements of 0.05 A from the lattice sites
    d = I.min_image(s.x - I.fcc_lattice(10, 10, 10, A), s.box, s.periodic)
    assert d.std() == pytest.approx(0.05, rel=0.05)
    # 3,000 K peak, sigma 8 A, at the box centre, on 300 K
    assert s.Te.min() >= 300.0 and s.Te.max() <= 3000.0
    c = I.min_image(s.x - 0.5 * s.box, s.box, s.periodic)
    r2 = (c * c).sum(axis=1)
    expect = 300.0 + 2700.0 * np.exp(-r2 / (2.0 * 64.0))
    assert np.allclose(s.Te, expect, rtol=1e-12)
    assert _kinetic_temperature(s) == pytest.approx(300.0, rel=0.06)
    assert np.allclose(s.v.mean(axis=0), 0.0, atol=1e-15)


def test_track_system_profile_and_size():
    s = I.track_system(10, 2)
    assert s.n == 4000
    # radial Gaussian about the z axis through the box centre: 20,000 K on the
    # axis (lattice sites lie on it), r0 = 2 nm, on 300 K
    rho = np.hypot(*I.min_image(s.x - 0.5 * s.box, s.box, s.periodic)[:, :2].T)
    on_axis = rho < 1e-9
    assert on_axis.any() and np.allclose(s.Te[on_axis], 20000.0)
    expect = 300.0 + 19700.0 * np.exp(-rho ** 2 / (2.0 * 400.0))
    assert np.allclose(s.Te, expect, rtol=1e-12)      # a function of rho only: no z dependence
    assert _kinetic_temperature(s) == pytest.approx(300.0, rel=0.06)


def test_laser_slab_surfaces_vacancies_and_depth():
    nxy, nz = 6, 20
    s = I.laser_slab_system(nxy, nz, 3)
    sites = 4 * nxy * nxy * nz
    assert s.n == sites - int(round(0.02 * sites))
    assert list(s.periodic) == [1, 1, 0]
    # 5 nm of vacuum below and above the film
    assert np.isclose(s.box[2], nz * A + 100.0)
    assert s.x[:, 2].min() >= 50.0 - 1e-12
    assert s.box[2] - s.x[:, 2].max() >= 50.0 + A / 2.0 - 1e-9
    # depth below the initial top surface
    assert s.depth.min() == 0.0 and np.allclose(s.depth, s.x[:, 2].max() - s.x[:, 2])
    assert np.all(s.Te == 300.0)
    # the full-size slab of the workload: 60 x 60 x 200 cells, 2 % of the sites empty
    full = 4 * 60 * 60 * 200
    assert full - int(round(0.02 * full)) == 2_822_400


def test_batch_replicas_sizes_and_hot_spots():
    reps = I.batch_replicas(12, 9, scale=0.02)
    for s in reps:
        c = round((s.n / 4) ** (1.0 / 3.0))
        assert s.n == 4 * c ** 3 and c >= 3
        # log-uniform in [8,000, 500,000] x scale, to the cubic cell count
        assert 4 * max(3, math.floor((8000 * 0.02 / 4) ** (1 / 3))) ** 3 <= s.n
        assert s.n <= 4 * math.ceil((500000 * 0.02 / 4) ** (1 / 3)) ** 3
        assert 300.0 <= s.Te.min() and s.Te.max() <= 30000.0
        assert s.Te.max() > 300.0
    assert len({s.n for s in reps}) > 3          # uneven sizes


@pytest.mark.parametrize("make", [
    lambda seed: I.track_system(6, seed),
    lambda seed: I.hot_spot_system(6, seed),
    lambda seed: I.laser_slab_system(4, 6, seed),
])
def test_generators_are_seeded(make):
    a, b, c = make(5), make(5), make(6)
    for f in ("x", "v", "Te"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(a.v, c.v)
