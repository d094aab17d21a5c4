"""FP64 CPU reference of the learned corrector network (test infrastructure).

The corrector is a two-layer message-passing network over the neighbour list
(node width 64) that adds a learned pair flux to the result Y of a window of
the propagator, so that the corrected window follows the plain substeps of
Eq. HeatTransport more closely.  Its only output is a pair flux, odd under
i <-> j, so sum_i T_i is kept exactly:

  inputs     delta_i = (Y_i - Tref) / Tmax,  D_ij = (delta_j - delta_i) / sigma,
             node features f_i = [Y_i / 1e4, T_l,i / 1e3 (0 below the kinetic-energy guard), z_i / 18]
             (z_i the neighbour count), edge features e_ij = [q_ij, rho_ij] with
             q_ij = D_ij^2 / (1 + D_ij^2) and rho_ij = r_ij / r_c (both symmetric)
  layer 1    mean-aggregated messages of the neighbours and their edges:
             in_i = [f_i, <f_j>, <q>, <q^2>, <rho>, <q rho>, 1, 0 x 5]       (16; <.> = mean over j)
             h1_i = relu(W1 in_i + b1),  h2_i = relu(W2 h1_i + b2),  u_i = W3 h2_i   (64, 64, 16)
  layer 2    edge MLP on the gathered node states:
             z_ij = u_i + u_j + P e_ij + b4,   g_ij = w4 . relu(z_ij)      (16 -> 1, symmetric)
  output     Y^_i = Y_i + kappa sum_j (Y_j - Y_i) g_ij,  kappa = n_w dt K  (the window's rate)

With w4 = 0 the corrector is the identity (the window itself).  Loss of a
window: L = (1/N) sum_i ((Y^_i - T*_i) / T*_i)^2 against the plain substeps T*.

Parameter vector (6336): [W1 (64 x 16) | b1 (64) | W2 (64 x 64) | b2 (64) |
W3 (16 x 64) | P (16 x 2) | b4 (16) | w4 (16)], matrices row-major (out x in).
Pinned by central finite differences, the identity at w4 = 0, the exact
conservation of sum_i Y_i and the symmetry of g (tests/test_oracle_gnn.py).
"""
from __future__ import annotations

import numpy as np

H = 64       # node width
U = 16       # edge width (projection of the node state gathered per edge)
F_IN = 16    # layer-1 input width (11 used)
SIZES = (("W1", (H, F_IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (U, H)),
         ("P", (U, 2)), ("b4", (U,)), ("w4", (U,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def init_params(seed: int = 0) -> np.ndarray:
    """He-scaled random layer weights, w4 = 0 (the identity corrector)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(N_PARAMS)
    w = unpack(p)
    w["W1"][:, :11] = rng.normal(0, np.sqrt(2.0 / 11), size=(H, 11))
    w["W2"][:] = rng.normal(0, np.sqrt(2.0 / H), size=(H, H))
    w["W3"][:] = rng.normal(0, np.sqrt(1.0 / H), size=(U, H))
    w["P"][:] = rng.normal(0, 0.5, size=(U, 2))
    w["b1"][:] = 0.05
    w["b2"][:] = 0.05
    return p


def _edges(rowptr, col):
    n = rowptr.shape[0] - 1
    i = np.repeat(np.arange(n), np.diff(rowptr))
    return i, col.astype(np.int64)


def features(Y, Tl, chi, rowptr, col, r, *, Tref, Tmax, sigma, rc):
    """Layer-1 inputs in [N, 16], edge features (q, rho) [E] and D [E]."""
    n = Y.shape[0]
    i, j = _edges(rowptr, col)
    z = np.diff(rowptr).astype(np.float64)
    delta = (Y - Tref) / Tmax
    D = (delta[j] - delta[i]) / sigma
    q = D * D / (1.0 + D * D)
    rho = r / rc
    f = np.stack([Y / 1.0e4, np.where(chi != 0, Tl / 1.0e3, 0.0), z / 18.0], axis=1)
    inv = np.where(z > 0, 1.0 / np.maximum(z, 1.0), 0.0)

    def mean(vals):
        s = np.zeros((n,) + vals.shape[1:])
        np.add.at(s, i, vals)
        return s * (inv[:, None] if s.ndim == 2 else inv)

    inp = np.zeros((n, F_IN))
    inp[:, 0:3] = f
    inp[:, 3:6] = mean(f[j])
    inp[:, 6] = mean(q)
    inp[:, 7] = mean(q * q)
    inp[:, 8] = mean(rho)
    inp[:, 9] = mean(q * rho)
    inp[:, 10] = 1.0
    return inp, q, rho, D


def forward(p, Y, Tl, chi, rowptr, col, r, *, Tref, Tmax, sigma, rc, kappa):
    """Corrected window result Y^ (FP64) and the intermediates of the backward."""
    w = unpack(p)
    i, j = _edges(rowptr, col)
    inp, q, rho, D = features(Y, Tl, chi, rowptr, col, r, Tref=Tref, Tmax=Tmax, sigma=sigma, rc=rc)
    a1 = inp @ w["W1"].T + w["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(a2, 0.0)
    u = h2 @ w["W3"].T
    ze = u[i] + u[j] + q[:, None] * w["P"][None, :, 0] + rho[:, None] * w["P"][None, :, 1] + w["b4"]
    re = np.maximum(ze, 0.0)
    g = re @ w["w4"]
    dY = Y[j] - Y[i]
    corr = np.zeros_like(Y)
    np.add.at(corr, i, dY * g)
    Yhat = Y + kappa * corr
    cache = dict(i=i, j=j, inp=inp, q=q, rho=rho, a1=a1, h1=h1, a2=a2, h2=h2, u=u, ze=ze, re=re, g=g, dY=dY)
    return Yhat, cache


def loss_and_grad(p, Y, Tstar, Tl, chi, rowptr, col, r, *, Tref, Tmax, sigma, rc, kappa):
    """Window loss L = mean(((Y^ - T*) / T*)^2) and its gradient in p (FP64)."""
    w = unpack(p)
    Yhat, c = forward(p, Y, Tl, chi, rowptr, col, r, Tref=Tref, Tmax=Tmax, sigma=sigma, rc=rc, kappa=kappa)
    n = Y.shape[0]
    rel = (Yhat - Tstar) / Tstar
    L = float((rel * rel).mean())
    G = 2.0 * rel / (Tstar * n)                      # dL / dY^_i
    i, j = c["i"], c["j"]
    grad = np.zeros_like(p)
    gw = unpack(grad)
    # every directed edge (i, j) of row i carries the term kappa dY_ij g_ij of Y^_i
    dg = kappa * c["dY"] * G[i]
    gw["w4"][:] = dg @ c["re"]
    dz = (dg[:, None] * w["w4"][None, :]) * (c["ze"] > 0)
    gw["P"][:, 0] = dz.T @ c["q"]
    gw["P"][:, 1] = dz.T @ c["rho"]
    gw["b4"][:] = dz.sum(0)
    du = np.zeros((n, U))
    np.add.at(du, i, dz)
    np.add.at(du, j, dz)
    gw["W3"][:] = du.T @ c["h2"]
    da2 = (du @ w["W3"]) * (c["a2"] > 0)
    gw["W2"][:] = da2.T @ c["h1"]
    gw["b2"][:] = da2.sum(0)
    da1 = (da2 @ w["W2"]) * (c["a1"] > 0)
    gw["W1"][:] = da1.T @ c["inp"]
    gw["b1"][:] = da1.sum(0)
    return L, grad, Yhat


def pair_distances(x, box, periodic, rowptr, col):
    """r_ij [E] of the list entries: minimum-image distances of the positions on
    the 2^-20 A grid of the neighbour search (the oracle's own quantisation)."""
    from . import quantize
    q, Lq = quantize(x, box, periodic)
    i, j = _edges(rowptr, col)
    d = q[j].astype(np.int64) - q[i].astype(np.int64)
    per = np.asarray(periodic) != 0
    for k in range(3):
        if per[k]:
            L = int(Lq[k])
            d[:, k] = np.where(2 * d[:, k] > L, d[:, k] - L, np.where(2 * d[:, k] < -L, d[:, k] + L, d[:, k]))
    d2 = (d * d).sum(1).astype(np.float64)
    return np.sqrt(d2) * 2.0 ** -20
