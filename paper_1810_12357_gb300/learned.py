"""Training and evaluation of the learned window propagators: the message-
passing network (ehc_nn_*) and the Chebyshev window with trained stage
coefficients (ehc_cheb_train_step).

Training windows come from the plain method itself: a context runs n_w
explicit substeps of Eq. HeatTransport with the coupling switched off (G = 0),
and each (state, state n_w substeps later) pair is one window.  The network is
Both are trained on the GPU by the library's own forward/backward kernels and Adam.
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
