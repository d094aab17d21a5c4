"""FP64 CPU reference of the learned 16-substep propagator (test infrastructure).

The network stands in for a window of n_w explicit substeps of Eq. HeatTransport
(flux part) on the same neighbour graph.  Two message-passing layers, hidden
width H, every pair term odd in the temperature difference so that the
predicted pair fluxes are antisymmetric and conserve sum_i T_i exactly:

  theta_i = T_i / Tmax,  D_ij = (theta_j - theta_i) / sigma,  q_ij = D_ij^2 / (1 + D_ij^2),
  s_ij = theta_i + theta_j
  layer 1 (edge -> node):  a_ij = relu(W1 [q_ij, s_ij] + b1),   h_i = sum_j D_ij a_ij      (R^H)
  layer 2 (edge flux):     phi_ij = D_ij (c0 + w . relu(W2 [q_ij, s_ij] + b2)) + u . (h_j - h_i)
  output:                  T^_i = T_i + (sigma Tmax) kappa sum_j phi_ij,   kappa = n_w dt K

With c0 = 1 and w = u = 0 the prediction is one Euler step of length n_w dt.
Loss of a window: L = (1/N) sum_i ((T^_i - T*_i) / (sigma Tmax))^2.

Parameter vector (8H + 1): [W1 (H x 2) | b1 (H) | W2 (H x 2) | b2 (H) | w (H) | u (H) | c0].
Pinned by central finite differences (tests/test_oracle_nn.py).  Parity with
the GPU kernels: forward and gradients (tests/test_gpu_nn.py).
"""
from __future__ import annotations

import numpy as np


def n_params(H: int) -> int:
    return 8 * H + 1


def unpack(p: np.ndarray, H: int):
    o = 0
    W1 = p[o:o + 2 * H].reshape(H, 2); o += 2 * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + 2 * H].reshape(H, 2); o += 2 * H
    b2 = p[o:o + H]; o += H
    w = p[o:o + H]; o += H
    u = p[o:o + H]; o += H
    c0 = p[o]
    return W1, b1, W2, b2, w, u, c0


def init_params(H: int, seed: int = 0) -> np.ndarray:
    """c0 = 1 (the one-Euler-step propagator), small random hidden weights."""
    rng = np.random.default_rng(seed)
    p = np.zeros(n_params(H))
    W1, b1, W2, b2, w, u, _ = unpack(p, H)
    W1[:] = rng.normal(0, 0.3, size=W1.shape)
    b1[:] = 0.1
    W2[:] = rng.normal(0, 0.3, size=W2.shape)
    b2[:] = 0.1
    w[:] = rng.normal(0, 0.01, size=H)
    u[:] = rng.normal(0, 0.01, size=H)
    p[-1] = 1.0
    return p


def _edges(rowptr, col):
    n = rowptr.shape[0] - 1
    i = np.repeat(np.arange(n), np.diff(rowptr))
    return i, col.astype(np.int64)


def forward(p, H, T, rowptr, col, *, Tmax, sigma, kappa):
    """Predicted temperatures T^ (FP64) and the intermediates of the backward."""
    W1, b1, W2, b2, w, u, c0 = unpack(p, H)
    th = T / Tmax
    i, j = _edges(rowptr, col)
    D = (th[j] - th[i]) / sigma
    q = D * D / (1.0 + D * D)
    s = th[i] + th[j]
    z1 = q[:, None] * W1[None, :, 0] + s[:, None] * W1[None, :, 1] + b1[None, :]
    a1 = np.maximum(z1, 0.0)
    h = np.zeros((T.shape[0], H))
    np.add.at(h, i, D[:, None] * a1)
    z2 = q[:, None] * W2[None, :, 0] + s[:, None] * W2[None, :, 1] + b2[None, :]
    a2 = np.maximum(z2, 0.0)
    phi = D * (c0 + a2 @ w) + (h[j] - h[i]) @ u
    F = np.zeros(T.shape[0])
    np.add.at(F, i, phi)
    scale = sigma * Tmax * kappa
    That = T + scale * F
    cache = dict(i=i, j=j, D=D, q=q, s=s, z1=z1, a1=a1, h=h, z2=z2, a2=a2, scale=scale)
    return That, cache


def loss_and_grad(p, H, T, Tstar, rowptr, col, *, Tmax, sigma, kappa):
    """Window loss and its gradient with respect to p (FP64)."""
    W1, b1, W2, b2, w, u, c0 = unpack(p, H)
    That, c = forward(p, H, T, rowptr, col, Tmax=Tmax, sigma=sigma, kappa=kappa)
    n = T.shape[0]
    Ts = sigma * Tmax
    r = (That - Tstar) / Ts
    L = float((r * r).mean())
    G = 2.0 * r / (n * Ts)                     # dL / dT^_i
    i, j, D, q, s = c["i"], c["j"], c["D"], c["q"], c["s"]
    gphi = G[i] * c["scale"]                    # dL / dphi_ij
    grad = np.zeros_like(p)
    gW1, gb1, gW2, gb2, gw, gu, _ = unpack(grad, H)
    # layer 2
    grad[-1] = float((gphi * D).sum())
    gw[:] = (gphi * D) @ c["a2"]
    m2 = (c["z2"] > 0).astype(float) * w[None, :] * (gphi * D)[:, None]
    gW2[:, 0] = (m2 * q[:, None]).sum(0)
    gW2[:, 1] = (m2 * s[:, None]).sum(0)
    gb2[:] = m2.sum(0)
    gu[:] = gphi @ (c["h"][j] - c["h"][i])
    # dL/dh_m = u * (sum_{i: m in N(i)} gphi_i - deg(m) gphi_m), lists are symmetric
    gh = np.zeros((n, H))
    np.add.at(gh, j, gphi[:, None] * u[None, :])
    np.add.at(gh, i, -gphi[:, None] * u[None, :])
    # layer 1: h_m = sum_j D_mj relu(z1_mj)
    m1 = gh[i] * (c["z1"] > 0) * D[:, None]
    gW1[:, 0] = (m1 * q[:, None]).sum(0)
    gW1[:, 1] = (m1 * s[:, None]).sum(0)
    gb1[:] = m1.sum(0)
    return L, grad, That
