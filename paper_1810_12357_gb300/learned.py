"""Training and evaluation of the learned window propagators: the message-
passing network (ehc_nn_*) and the Chebyshev window with trained stage
coefficients (ehc_cheb_train_step).

Training windows come from the plain method itself: a context runs n_w
explicit substeps of Eq. HeatTransport with the coupling switched off (G = 0),
and each (state, state n_w substeps later) pair is one window; rollouts chain
several windows of one trajectory.  Both propagators are trained on the GPU by
the library's own forward/backward kernels and Adam.
"""
from __future__ import annotations

import numpy as np

from . import Ehc


def generate_windows(system, params: dict, n_windows: int, n_w: int = 16, stride: int = 1):
    """(T_in, T_out) device tensor pairs from a frozen-atom, flux-only run of the
    plain method (caller order).  `stride` windows are skipped between samples."""
    import torch
    p = dict(params, G=0.0, frozen=1)
    g = Ehc(p, system)
    g.set_te(system.Te)
    x = torch.as_tensor(system.x, device="cuda")
    v = torch.as_tensor(system.v, device="cuda")
    g.build_neighbors(x, v)
    pairs = []
    for w in range(n_windows):
        for _ in range(stride - 1):
            g.substep(n_w)
        t0 = g.get_te()
        g.substep(n_w)
        t1 = g.get_te()
        pairs.append((t0, t1))
    return g, pairs


def train(model, pairs, steps: int, lr: float = 3e-3, log_every: int = 0, ctx=None, **kw):
    """Adam steps cycling through the windows of the network (EhcNN) or of the
    trained Chebyshev window (EhcCheb); returns the loss history.  `ctx` is the
    context the windows were generated on (default the model's own); further
    keywords go to the model's train_step."""
    hist = []
    for k in range(steps):
        t0, t1 = pairs[k % len(pairs)]
        loss = model.train_step(t0, t1, lr, ctx=ctx, **kw)
        hist.append(loss)
        if log_every and k % log_every == 0:
            print(f"step {k} loss {loss:.4e}")
    return hist


def window_error(model, pairs, ctx=None):
    """Max relative and RMS absolute error of flux-only predictions on windows."""
    import torch
    mx, ms = 0.0, 0.0
    for t0, t1 in pairs:
        p = model.predict(t0) if ctx is None else model.predict(t0, ctx=ctx)
        d = (p - t1).abs()
        mx = max(mx, float((d / t1).max()))
        ms = max(ms, float(torch.sqrt((d * d).mean())))
    return mx, ms


def init_params(H: int, seed: int = 0) -> np.ndarray:
    """c0 = 1 (one Euler step of the whole window), small hidden weights."""
    rng = np.random.default_rng(seed)
    p = np.zeros(8 * H + 1, dtype=np.float32)
    p[0:2 * H] = rng.normal(0, 0.3, size=2 * H)          # W1
    p[2 * H:3 * H] = 0.1                                  # b1
    p[3 * H:5 * H] = rng.normal(0, 0.3, size=2 * H)      # W2
    p[5 * H:6 * H] = 0.1                                  # b2
    p[6 * H:7 * H] = rng.normal(0, 0.01, size=H)         # w
    p[7 * H:8 * H] = rng.normal(0, 0.01, size=H)         # u
    p[8 * H] = 1.0                                        # c0
    return p


def generate_trajectory(system, params: dict, n_windows: int, n_w: int = 100, skip: int = 1):
    """A plain flux-only trajectory for rollout training: the state after `skip`
    windows of n_w plain substeps (the sharp initial front is left to the
    residual test) and the states after each of the next n_windows windows, as
    (context, T0, targets [n_windows, N]) on the device, caller order."""
    import torch
    p = dict(params, G=0.0, frozen=1)
    g = Ehc(p, system)
    g.set_te(system.Te)
    x = torch.as_tensor(system.x, device="cuda")
    v = torch.as_tensor(system.v, device="cuda")
    g.build_neighbors(x, v)
    for _ in range(skip):
        g.substep(n_w)
    t0 = g.get_te()
    targets = []
    for _ in range(n_windows):
        g.substep(n_w)
        targets.append(g.get_te())
    return g, t0, torch.stack(targets).contiguous()


def rollout_error(model, t0, targets, ctx=None):
    """Max relative error after each window when the model's windows are chained
    from t0 (flux only), against the plain trajectory."""
    out = []
    t = t0
    for k in range(targets.shape[0]):
        t = model.predict(t) if ctx is None else model.predict(t, ctx=ctx)
        out.append(float(((t - targets[k]).abs() / targets[k]).max()))
    return out


def train_rollout(model, data, steps: int, lr: float = 3e-3, power: int = 8, lr_final: float | None = None):
    """Adam steps on the rollout loss, cycling through data = [(ctx, t0, targets)];
    the rate drops to lr_final for the last quarter.  Returns the loss history."""
    hist = []
    for k in range(steps):
        ctx, t0, tt = data[k % len(data)]
        rate = lr if (lr_final is None or k < steps * 3 // 4) else lr_final
        hist.append(model.train_rollout(t0, tt, rate, ctx=ctx, power=power))
    return hist


def train_track_window(n_w: int = 100, stages: int = 15, damping: float = 2.0 / 13.0, order: int = 2,
                       train_steps: int = 400, power: int = 2, nwin: int = 6):
    """Stage coefficients of the learned window for the swift-ion track: Adam on
    rollouts of `nwin` chained windows against the plain method's trajectories
    (coupling off) of 256,000-atom track and hot-spot cells (40^3 cells), from the
    damped Chebyshev values of the given order, each rollout started after the
    first window (the sharp initial front is left to the residual test).  Returns
    the coefficients (nu, mut, kap, gam) and a record of the training with
    held-out rollout errors of a seventh cell."""
    import time
    from . import EhcCheb
    from . import inputs as I
    p = I.params_track()
    t0 = time.perf_counter()
    train_sys = [I.track_system(40, 100 + k, peak=8000.0 + 6000.0 * k, r0=12.0 + 4.0 * k) for k in range(3)]
    train_sys += [I.hot_spot_system(40, 150 + k, peak=6000.0 + 6000.0 * k, sigma=8.0 + 3.0 * k, disp_sigma=0.0)
                  for k in range(3)]
    data = [generate_trajectory(s, p, nwin, n_w) for s in train_sys]
    w = EhcCheb(data[0][0], n_w, stages, damping, order=order)
    beta0 = w.stability()
    # the stability range of training: the spectrum of the training states
    spec = max(w.spectrum(t_in, iters=300, ctx=c) for c, t_in, _ in data)
    hist = train_rollout(w, data, train_steps, lr=5e-3, lr_final=2e-3, power=power)
    coeffs = [c.copy() for c in w.coefficients()]
    t_train = time.perf_counter() - t0
    del data
    # held-out rollouts of another track: trained against untrained coefficients
    hc, h0, ht = generate_trajectory(I.track_system(40, 199, peak=20000.0, r0=20.0), p, nwin, n_w)
    base = EhcCheb(hc, n_w, stages, damping, order=order)
    per_u = rollout_error(base, h0, ht, ctx=hc)
    per_t = rollout_error(w, h0, ht, ctx=hc)
    info = {"train_s": t_train, "train_rollouts": len(train_sys), "rollout_windows": nwin,
            "train_steps": train_steps,
            "train_cells": "256,000-atom tracks and hot spots (40^3 cells), rollouts from the end of the first window",
            "start": "damped Chebyshev order %d, damping %.4g" % (order, damping),
            "loss": "sum over the rollout's windows of mean relative error^%d" % power,
            "training_spectrum_tauK_lambda_max": spec, "stability_untrained": beta0,
            "stability_trained": w.stability(), "loss_first": hist[0], "loss_last": hist[-1],
            "heldout_256k_rollout_max_rel_err_per_window": {"trained": per_t, "untrained": per_u}}
    return coeffs, info


def corrector_init(seed: int = 0):
    """Initial corrector parameters (6336, FP32): He-scaled node layers, w4 = 0,
    so that the untrained corrector is the identity."""
    import numpy as np
    rng = np.random.default_rng(seed)
    H, U, F = 64, 16, 16
    W1 = np.zeros((H, F))
    W1[:, :11] = rng.normal(0, np.sqrt(2.0 / 11), size=(H, 11))
    W2 = rng.normal(0, np.sqrt(2.0 / H), size=(H, H))
    W3 = rng.normal(0, np.sqrt(1.0 / H), size=(U, H))
    P = rng.normal(0, 0.5, size=(U, 2))
    parts = [W1.ravel(), np.full(H, 0.05), W2.ravel(), np.full(H, 0.05), W3.ravel(), P.ravel(), np.zeros(U),
             np.zeros(U)]
    return np.concatenate(parts).astype(np.float32)


def corrector_windows(system, params: dict, coeffs, n_windows: int, n_w: int = 100, stages: int = 15,
                      order: int = 2, skip: int = 1):
    """Training pairs of the corrector from one cell: the states a run of the
    window propagator visits (the initial state, or the plain state after `skip`
    windows, then the window's own chained results) and, from each, the window's
    result Y and the n_w plain substeps' result T* (coupling off), as
    (context, [(Y, T*)], kappa)."""
    import torch
    from . import EhcCheb
    p = dict(params, G=0.0, frozen=1)
    g = Ehc(p, system)
    g.set_te(system.Te)
    x = torch.as_tensor(system.x, device="cuda")
    v = torch.as_tensor(system.v, device="cuda")
    g.build_neighbors(x, v)
    if skip:
        g.substep(skip * n_w)
    w = EhcCheb(g, n_w, stages, 2.0 / 13.0, order=order)
    w.set_coefficients(*coeffs)
    s = g.get_te()
    pairs = []
    for _ in range(n_windows):
        y = w.predict(s)
        g.set_te(s)
        g.build_neighbors(x, v)     # set_te starts a new MD step (frozen atoms: the same list)
        g.substep(n_w)
        pairs.append((y, g.get_te()))
        s = y
    return g, pairs, w.kappa()


def train_track_corrector(coeffs, n_w: int = 100, stages: int = 15, order: int = 2, steps: int = 800,
                          lr: float = 3e-4, n_windows: int = 24, seed: int = 0, cells: int = 60, skip: int = 1):
    """The corrector network of the learned window on the swift-ion track: Adam on
    (window result, plain substeps) pairs of six track and hot-spot cells
    (`cells`^3 FCC cells, 864,000 atoms at 60), taken on the states a run of the
    window with the given stage coefficients visits after the first `skip`
    windows (n_windows windows).  Returns the parameters and a record with the
    held-out error of a seventh cell's windows with and without the corrector."""
    import time
    import numpy as np
    from . import EhcGnn
    from . import inputs as I
    p = I.params_track()
    t0 = time.perf_counter()
    nc = cells
    cells = [I.track_system(nc, 100 + k, peak=8000.0 + 6000.0 * k, r0=12.0 + 4.0 * k) for k in range(3)]
    cells += [I.hot_spot_system(nc, 150 + k, peak=6000.0 + 6000.0 * k, sigma=8.0 + 3.0 * k, disp_sigma=0.0)
              for k in range(3)]
    data = [corrector_windows(c, p, coeffs, n_windows, n_w, stages, order, skip=skip) for c in cells]
    net = EhcGnn(data[0][0], params=corrector_init(seed))
    hist = []
    for k in range(steps):
        ctx, pairs, kappa = data[k % len(data)]
        y, ts = pairs[(k // len(data)) % len(pairs)]
        hist.append(net.train_step(y, ts, kappa, lr if k < 3 * steps // 4 else 0.3 * lr, ctx=ctx))
    params = net.get_params()
    t_train = time.perf_counter() - t0
    del data
    # held-out: the windows of a seventh track, without and with the corrector
    hc, hp, hk = corrector_windows(I.track_system(nc, 199, peak=20000.0, r0=20.0), p, coeffs, n_windows, n_w,
                                   stages, order, skip=skip)
    hnet = EhcGnn(hc, params=params)
    err_u = [float(((y - t).abs() / t).max()) for y, t in hp]
    err_t = [float(((hnet.apply(y, hk) - t).abs() / t).max()) for y, t in hp]
    info = {"train_s": t_train, "train_cells": f"{len(cells)} cells of {nc}^3 FCC cells", "windows_per_cell": n_windows,
            "train_steps": steps,
            "loss_first": hist[0], "loss_last": hist[-1],
            "heldout_256k_window_max_rel_err": {"window": err_u, "window_and_corrector": err_t}}
    return params, info
