"""Learned window propagator: GPU forward and gradients against the FP64 CPU
reference (oracle/nn.py) with the same BF16-rounded weights, training on
windows of the plain method, and the residual-triggered fallback."""
import numpy as np
import pytest

import oracle
from oracle import nn as onn
from paper_1810_12357_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _bf16(p):
    import torch
    return torch.as_tensor(p, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def _setup(H=8, cells=4, seed=11):
    import torch
    from paper_1810_12357_gb300 import Ehc, EhcNN
    s = I.hot_spot_system(cells, seed, peak=2500.0, sigma=5.0)
    p = dict(I.params_hotspot_fp64(), flux_prec=0, G=0.0)
    g = Ehc(p, s)
    g.set_te(s.Te)
    g.build_neighbors(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.v, device="cuda"))
    K = g.energy()["K_per_fs"]
    net = EhcNN(g, hidden=H, n_window=16, sigma=0.02)
    rp, col = oracle.neighbors(s.x, s.box, s.periodic, p["rc"])
    kappa = 16 * p["dt_sub"] * K
    return s, p, g, net, rp, col, kappa


@pytest.mark.parametrize("H", [8, 16])
def test_forward_and_gradient_match_fp64_reference(H):
    import torch
    s, p, g, net, rp, col, kappa = _setup(H)
    prm = onn.init_params(H, 5)
    prm[-1 - 2 * H:-1] = np.random.default_rng(6).normal(0, 0.3, size=2 * H)
    net.set_params(prm.astype(np.float32))
    pb = _bf16(prm.astype(np.float32))
    Tin = torch.as_tensor(s.Te, device="cuda")
    Tstar = s.Te + np.random.default_rng(7).normal(0, 20.0, size=s.n)
    loss, grad = net.train_step(Tin, torch.as_tensor(Tstar, device="cuda"), 0.0, want_grad=True)
    L, g_ref, That = onn.loss_and_grad(pb, H, s.Te, Tstar, rp, col, Tmax=p["Tmax"], sigma=0.02, kappa=kappa)
    assert loss == pytest.approx(L, rel=2e-2)
    cos = float(grad @ g_ref / (np.linalg.norm(grad) * np.linalg.norm(g_ref)))
    assert cos > 0.999, cos
    big = np.abs(g_ref) > 1e-3 * np.abs(g_ref).max()
    assert np.max(np.abs(grad[big] - g_ref[big]) / np.abs(g_ref[big])) < 2e-2
    pred = net.predict(Tin).cpu().numpy()
    inc_g, inc_r = pred - s.Te, That - s.Te
    assert np.max(np.abs(inc_g - inc_r)) < 2e-2 * np.max(np.abs(inc_r)) + 1e-6


def test_training_beats_the_untrained_window_step():
    # windows of 16 substeps from the plain method (coupling off); held-out windows
    from paper_1810_12357_gb300 import EhcNN, learned
    s = I.track_system(12, 21, r0=9.0, peak=8000.0)
    p = dict(I.params_track(), Tmax=2e4)
    g, pairs = learned.generate_windows(s, p, 24, 16)
    net = EhcNN(g, hidden=8, n_window=16, sigma=0.02, params=learned.init_params(8, 1))
    train, test = pairs[:16], pairs[16:]
    e0 = learned.window_error(net, test)
    hist = learned.train(net, train, 400, lr=3e-3)
    e1 = learned.window_error(net, test)
    assert hist[-1] < 0.5 * hist[0]
    assert e1[1] < 0.5 * e0[1], (e0, e1)
    assert e1[0] < 1e-2


def test_step_falls_back_to_plain_substeps():
    # with tau = 0 every window is redone by the plain method: identical to a plain run
    import torch
    from paper_1810_12357_gb300 import Ehc, EhcNN, learned
    s = I.track_system(8, 22, r0=6.0)
    p = I.params_track()
    a = Ehc(p, s)
    b = Ehc(p, s)
    for c in (a, b):
        c.set_te(s.Te)
    x = torch.as_tensor(s.x, device="cuda")
    v = torch.as_tensor(s.v, device="cuda")
    a.build_neighbors(x, v)
    b.build_neighbors(x, v)
    net = EhcNN(a, hidden=8, n_window=16, sigma=1e-3, params=learned.init_params(8, 2))
    for w in range(3):
        fb, rho = net.step(0.0)
        assert fb
        b.substep(16)
    assert np.array_equal(a.get_te().cpu().numpy(), b.get_te().cpu().numpy())
    # an accepted window keeps the energy ledger closed
    fb, rho = net.step(1e9)
    assert not fb
    a.couple(v, 16 * p["dt_sub"])
    assert abs(a.energy()["drift"]) < 1e-8
