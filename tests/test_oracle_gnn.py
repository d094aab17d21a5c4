"""Pins of the FP64 corrector network (oracle/gnn.py) against what its
definition fixes: the gradient against central differences of the forward,
the identity at w4 = 0, exact conservation of sum_i Y_i by the antisymmetric
pair flux, the symmetry of the pair coefficient g_ij, and the layer-1 inputs
of a perfect FCC lattice at a uniform temperature (closed form from the shell
geometry)."""
import math

import numpy as np
import pytest

import oracle
from oracle import gnn
from paper_1810_12357_gb300 import inputs as I

KW = dict(Tref=300.0, Tmax=1.0e5, sigma=1.0e-3, rc=4.0)


def _graph(n_cells=3, seed=3):
    s = I.hot_spot_system(n_cells, seed, peak=6000.0, sigma=4.0, disp_sigma=0.08)
    rp, col = oracle.neighbors(s.x, s.box, s.periodic, 4.0, cap_per_atom=40)
    r = gnn.pair_distances(s.x, s.box, s.periodic, rp, col)
    rng = np.random.default_rng(seed)
    Tl = rng.uniform(250.0, 350.0, s.n)
    chi = (rng.uniform(size=s.n) > 0.1).astype(np.uint8)
    return s, rp, col, r, Tl, chi


def _params(seed=1):
    p = gnn.init_params(seed)
    w = gnn.unpack(p)
    rng = np.random.default_rng(seed + 7)
    w["w4"][:] = rng.normal(0, 0.3, gnn.U)
    w["b4"][:] = rng.normal(0, 0.3, gnn.U)
    return p


def test_gradient_matches_central_differences():
    s, rp, col, r, Tl, chi = _graph()
    p = _params()
    rng = np.random.default_rng(5)
    Tstar = s.Te * (1.0 + rng.normal(0, 0.01, s.n))
    kw = dict(KW, kappa=0.3)
    L, g, _ = gnn.loss_and_grad(p, s.Te, Tstar, Tl, chi, rp, col, r, **kw)
    # every parameter of the edge layer and a sample of each node-layer matrix
    off = np.cumsum([0] + [int(np.prod(sh)) for _, sh in gnn.SIZES])
    idx = list(range(off[5], off[8]))
    for k in range(5):
        idx += list(rng.choice(np.arange(off[k], off[k + 1]), size=min(40, off[k + 1] - off[k]), replace=False))
    worst = 0.0
    for m in idx:
        h = 1e-6 * max(1.0, abs(p[m]))
        pp, pm = p.copy(), p.copy()
        pp[m] += h
        pm[m] -= h
        Lp = gnn.loss_and_grad(pp, s.Te, Tstar, Tl, chi, rp, col, r, **kw)[0]
        Lm = gnn.loss_and_grad(pm, s.Te, Tstar, Tl, chi, rp, col, r, **kw)[0]
        fd = (Lp - Lm) / (2 * h)
        worst = max(worst, abs(fd - g[m]) / (abs(g[m]) + 1e-3 * np.abs(g).max()))
    assert worst < 1e-5, worst


def test_identity_at_zero_output_weights_and_conservation():
    s, rp, col, r, Tl, chi = _graph(seed=4)
    p = gnn.init_params(2)
    Y0, _ = gnn.forward(p, s.Te, Tl, chi, rp, col, r, kappa=0.3, **KW)
    assert np.array_equal(Y0, s.Te)
    p = _params(3)
    Y, c = gnn.forward(p, s.Te, Tl, chi, rp, col, r, kappa=0.3, **KW)
    assert np.abs(Y - s.Te).max() > 1e-3
    assert float(Y.sum()) == pytest.approx(float(s.Te.sum()), rel=1e-13)
    # the pair coefficient is symmetric: g_ij = g_ji
    i, j, g = c["i"], c["j"], c["g"]
    lookup = {(a, b): v for a, b, v in zip(i.tolist(), j.tolist(), g.tolist())}
    assert all(abs(lookup[(b, a)] - v) <= 1e-12 * (1 + abs(v)) for (a, b), v in lookup.items())


def test_layer1_inputs_of_a_uniform_perfect_lattice():
    # perfect FCC Cu, uniform Y: every atom has 12 neighbours at a/sqrt2 and 6 at a,
    # q = 0 on every edge, the neighbours' mean node features equal the atom's own
    a = I.CU_A
    x = I.fcc_lattice(4, 4, 4, a)
    box = np.array([4 * a] * 3)
    per = np.array([1, 1, 1], dtype=np.int32)
    rp, col = oracle.neighbors(x, box, per, 4.0, cap_per_atom=40)
    r = gnn.pair_distances(x, box, per, rp, col)
    n = x.shape[0]
    Y = np.full(n, 2500.0)
    Tl = np.full(n, 300.0)
    chi = np.ones(n, dtype=np.uint8)
    inp, q, rho, D = gnn.features(Y, Tl, chi, rp, col, r, **KW)
    rho_mean = (12 * (a / math.sqrt(2.0)) + 6 * a) / 18.0 / 4.0
    f = np.array([0.25, 0.3, 1.0])
    assert np.allclose(inp[:, 0:3], f, rtol=0, atol=1e-15)
    assert np.allclose(inp[:, 3:6], f, rtol=0, atol=1e-15)
    assert np.all(inp[:, 6:8] == 0.0) and np.all(inp[:, 9] == 0.0)
    assert np.allclose(inp[:, 8], rho_mean, rtol=2e-7)       # the 2^-20 A grid
    assert np.all(inp[:, 10] == 1.0) and np.all(inp[:, 11:] == 0.0)
    # an atom below the kinetic-energy guard reports no lattice temperature
    chi[5] = 0
    inp2 = gnn.features(Y, Tl, chi, rp, col, r, **KW)[0]
    assert inp2[5, 1] == 0.0 and inp2[5, 4] == pytest.approx(0.3, abs=1e-15)
