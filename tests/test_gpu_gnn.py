"""The corrector network on the GPU (ehc_gnn_*) against its FP64 reference
oracle/gnn.py: the correction of a window result (BF16 weights and
activations, FP32 accumulation on the tensor cores), the loss and its gradient,
the identity at zero weights, exact conservation of sum_i T_i, and training
that lowers a window's error."""
import numpy as np
import pytest

import oracle
from oracle import gnn
from paper_1810_12357_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SIGMA = 1.0e-3


def _bf16(p):
    """Round FP32/FP64 values to BF16 (nearest even), as the kernels hold the weights."""
    a = np.asarray(p, dtype=np.float32).copy()
    u = a.view(np.uint32)
    u += 0x7FFF + ((u >> 16) & 1)
    u &= 0xFFFF0000
    return a.astype(np.float64)


def _setup(seed=3, cells=7):
    import torch
    from paper_1810_12357_gb300 import Ehc
    s = I.hot_spot_system(cells, seed, peak=9000.0, sigma=6.0, disp_sigma=0.05)
    p = dict(I.params_track(), frozen=1)
    g = Ehc(p, s)
    g.set_te(s.Te)
    g.build_neighbors(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.v, device="cuda"))
    rp, col = g.export_neighbors(cap_per_atom=32)
    r = gnn.pair_distances(s.x, s.box, s.periodic, rp, col)
    Tl = g.get_lattice_temperature().cpu().numpy()
    chi = (Tl >= 0.0).astype(np.uint8)
    return s, p, g, rp, col, r, Tl, chi


def _params(seed):
    p = gnn.init_params(seed)
    w = gnn.unpack(p)
    rng = np.random.default_rng(seed + 11)
    w["w4"][:] = rng.normal(0, 0.3, gnn.U)
    w["b4"][:] = rng.normal(0, 0.3, gnn.U)
    return _bf16(p)


def _cos(a, b):
    return float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)))


def test_corrector_forward_matches_fp64_reference():
    import torch
    from paper_1810_12357_gb300 import EhcGnn
    s, p, g, rp, col, r, Tl, chi = _setup()
    prm = _params(1)
    net = EhcGnn(g, SIGMA, params=prm)
    kappa = 0.3
    Y = torch.as_tensor(s.Te, device="cuda")
    Yh, dY = net.apply(Y, kappa, want_dY=True)
    dYg = dY.cpu().numpy()
    Yo, c = gnn.forward(prm, s.Te, Tl, chi, rp, col, r, Tref=p["Tref"], Tmax=p["Tmax"], sigma=SIGMA, rc=p["rc"],
                        kappa=kappa)
    dYo = Yo - s.Te
    cos = _cos(dYg, dYo)
    err = float(np.abs(dYg - dYo).max() / np.abs(dYo).max())
    print(f"corrector forward: {s.n} atoms, max |dY| {np.abs(dYo).max():.3e} K, cosine {cos:.6f}, max err {err:.2e}")
    assert np.abs(dYo).max() > 1.0
    assert cos > 0.999 and err < 2e-2
    # the pair fluxes keep sum_i T_i; Y^ = Y + dY
    assert abs(float(dYg.sum())) < 1e-9 * float(np.abs(dYg).sum())
    assert np.allclose(Yh.cpu().numpy(), s.Te + dYg, rtol=0, atol=1e-9)


def test_corrector_zero_weights_is_the_identity():
    import torch
    from paper_1810_12357_gb300 import EhcGnn
    s, p, g, rp, col, r, Tl, chi = _setup(seed=4, cells=5)
    net = EhcGnn(g, SIGMA)
    Y = torch.as_tensor(s.Te, device="cuda")
    assert torch.equal(net.apply(Y, 0.3), Y)


def test_corrector_gradient_matches_fp64_reference():
    import torch
    from paper_1810_12357_gb300 import EhcGnn
    s, p, g, rp, col, r, Tl, chi = _setup(seed=5)
    prm = _params(2)
    net = EhcGnn(g, SIGMA, params=prm)
    rng = np.random.default_rng(9)
    Tstar = s.Te * (1.0 + rng.normal(0, 0.02, s.n))
    kappa = 0.3
    Lg, gg = net.train_step(torch.as_tensor(s.Te, device="cuda"), torch.as_tensor(Tstar, device="cuda"), kappa,
                            0.0, want_grad=True)
    Lo, go, _ = gnn.loss_and_grad(prm, s.Te, Tstar, Tl, chi, rp, col, r, Tref=p["Tref"], Tmax=p["Tmax"],
                                  sigma=SIGMA, rc=p["rc"], kappa=kappa)
    assert Lg == pytest.approx(Lo, rel=1e-3)
    off = np.cumsum([0] + [int(np.prod(sh)) for _, sh in gnn.SIZES])
    worst = 1.0
    for k, (name, _) in enumerate(gnn.SIZES):
        a, b = gg[off[k]:off[k + 1]].astype(np.float64), go[off[k]:off[k + 1]]
        if np.linalg.norm(b) == 0:
            continue
        cs = _cos(a, b)
        rel = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        print(f"gradient {name}: cosine {cs:.5f}, relative error {rel:.2e}")
        worst = min(worst, cs)
        assert cs > 0.99 and rel < 0.1, name
    tot = _cos(gg.astype(np.float64), go)
    assert tot > 0.999, tot


def test_training_lowers_the_window_error():
    # windows of the plain method (coupling off): the corrector is trained on
    # (window result, 100 plain substeps) pairs of two hot spots, on the states a
    # run of the second-order window visits, and lowers the error of the windows
    # of a third hot spot it has not seen
    import torch
    from paper_1810_12357_gb300 import Ehc, EhcCheb, EhcGnn, learned
    p = I.params_track()
    cells = [I.hot_spot_system(12, 60 + k, peak=9000.0 + 5000.0 * k, sigma=5.0 + 2.0 * k, disp_sigma=0.0)
             for k in range(3)]
    # the untrained second-order window's coefficients
    g0 = Ehc(dict(p, G=0.0, frozen=1), cells[0])
    g0.set_te(cells[0].Te)
    g0.build_neighbors(torch.as_tensor(cells[0].x, device="cuda"), torch.as_tensor(cells[0].v, device="cuda"))
    coeffs = EhcCheb(g0, 100, 15, 2.0 / 13.0, order=2).coefficients()
    data = [learned.corrector_windows(c, p, coeffs, 4) for c in cells]
    net = EhcGnn(data[0][0], params=learned.corrector_init(0))

    def held_out():
        ctx, pairs, kappa = data[2]
        return [float(((net.apply(y, kappa, ctx=ctx) - t).abs() / t).max()) for y, t in pairs]

    before = held_out()
    losses = []
    for it in range(400):
        ctx, pairs, kappa = data[it % 2]
        y, t = pairs[(it // 2) % len(pairs)]
        losses.append(net.train_step(y, t, kappa, 1e-3, ctx=ctx))
    after = held_out()
    print("corrector training: loss " + f"{np.mean(losses[:10]):.3e} -> {np.mean(losses[-10:]):.3e}; held-out "
          "window max errors " + ", ".join(f"{a:.2e} -> {b:.2e}" for a, b in zip(before, after)))
    assert np.mean(losses[-10:]) < 0.8 * np.mean(losses[:10])
    assert np.mean(after) < np.mean(before)
