"""Pins of the FP64 reference of the learned propagator: gradients against
central finite differences, exact conservation of sum T by the antisymmetric
pair fluxes, and the c0 = 1 network equal to one Euler step of the linearised
pair term."""
import numpy as np
import pytest

import oracle
from oracle import nn
from paper_1810_12357_gb300 import inputs as I


def _graph(seed=0, cells=3):
    s = I.hot_spot_system(cells, seed, peak=2500.0, sigma=4.0)
    rp, col = oracle.neighbors(s.x, s.box, s.periodic, 4.0)
    return s, rp, col


def test_gradient_matches_finite_differences():
    s, rp, col = _graph(1)
    H = 4
    p = nn.init_params(H, 3)
    p[nn.n_params(H) - 1 - 2 * H:-1] = np.random.default_rng(4).normal(0, 0.2, size=2 * H)   # w, u
    kw = dict(Tmax=2e4, sigma=0.02, kappa=0.05)
    Tstar = s.Te + np.random.default_rng(5).normal(0, 5.0, size=s.n)
    L, g, _ = nn.loss_and_grad(p, H, s.Te, Tstar, rp, col, **kw)
    eps = 1e-6
    for k in range(p.shape[0]):
        dp = np.zeros_like(p)
        dp[k] = eps
        Lp, _, _ = nn.loss_and_grad(p + dp, H, s.Te, Tstar, rp, col, **kw)
        Lm, _, _ = nn.loss_and_grad(p - dp, H, s.Te, Tstar, rp, col, **kw)
        fd = (Lp - Lm) / (2 * eps)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-12 * max(1.0, abs(L))), k


def test_pair_fluxes_conserve_sum_T():
    s, rp, col = _graph(2)
    H = 6
    p = nn.init_params(H, 7)
    p[-1 - 2 * H:-1] = np.random.default_rng(8).normal(0, 0.5, size=2 * H)
    That, _ = nn.forward(p, H, s.Te, rp, col, Tmax=2e4, sigma=0.02, kappa=0.05)
    assert abs(That.sum() - s.Te.sum()) / s.Te.sum() < 1e-14


def test_plain_network_is_one_euler_step_of_the_linear_term():
    # c0 = 1, w = u = 0: T^ = T + n_w dt K Tmax sum_j (theta_j - theta_i)
    s, rp, col = _graph(3)
    H = 4
    p = nn.init_params(H, 1)
    p[-1 - 2 * H:-1] = 0.0
    Tmax, kappa = 2e4, 0.05
    That, _ = nn.forward(p, H, s.Te, rp, col, Tmax=Tmax, sigma=0.02, kappa=kappa)
    i = np.repeat(np.arange(s.n), np.diff(rp))
    lap = np.zeros(s.n)
    np.add.at(lap, i, s.Te[col] - s.Te[i])
    assert np.allclose(That, s.Te + kappa * lap, rtol=1e-14, atol=1e-9)
