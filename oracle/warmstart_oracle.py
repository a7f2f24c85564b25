"""FP64 CPU oracle of the learned warm start: features from the compressed SVD, the per-row MLP
(forward, gradient, Adam), and the maps between network outputs and initial factors.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product path.

The paper initialises at random (Section 5, "random initialization"); the warm start is a
systems pattern on top of the method: NNDSVD (Boutsidis & Gallopoulos 2008) of the compressed
data, corrected row by row by a small network trained on solutions the compressed NMF itself
produces. Definitions (r components, X ~ Q_L X_hat with X_hat = U' S V^T, u_j = Q_L u'_j):

  mode_j       which sign part NNDSVD keeps: 0 = absolute value (j = 0), 1 = positive parts,
               2 = negative parts, 3 = none (both products zero)
  p(x)         that part of x (|x|, x+, x-, 0)
  W_b[:, j]    p(u_j) / ||p(u_j)||            (unit columns)
  H_b[j, :]    f_j^2 p(v_j) / ||p(v_j)||      f_j^2 = s_j ||p(u_j)|| ||p(v_j)|| (for j = 0 the
               norms are those of |u_0|, |v_0|, i.e. 1), so that W_b H_b is the NNDSVD product
  hscale_j     ||H_b[j, :]|| = f_j^2
  F_w[i]       [sqrt(m) c_j u_ij (j < r), sqrt(m) W_b[i, j] (j < r), s_j / s_0 (j < r)]
  F_h[c]       [sqrt(n) c_j v_cj, sqrt(n) H_b[j, c] / hscale_j, s_j / s_0]
               c_j = +1 (mode 1), -1 (mode 2); mode 0 uses |u_ij|, |v_cj|; mode 3 gives 0
  W_0          max(0, W_b + D_w / sqrt(m))            D_w = net_W(F_w)   (m x r)
  H_0          max(0, H_b + hscale * D_h^T / sqrt(n))  D_h = net_H(F_h)   (n x r)

Network: three layers, y = W3^T relu(W2^T relu(W1^T x + b1) + b2) + b3 with W1 (F x Hd),
W2 (Hd x Hd), W3 (Hd x r) stored row-major in one vector [W1, b1, W2, b2, W3, b3]. The weight
matrices take part in the arithmetic rounded to BF16 (round to nearest even); biases and
activations stay in full precision; the loss is the mean of squared errors over all outputs;
the gradient is that of the rounded weights (applied to the full-precision master copy).

Pins (tests/test_oracle_pins.py): central finite differences of the loss; Adam's first step
closed form; a zero last layer reproduces the NNDSVD factors; W_b H_b equals the NNDSVD product
of nndsvd_compressed; unit columns of W_b.
"""
from __future__ import annotations

import numpy as np

from .nmf_oracle import _neg, _pos

__all__ = ["bf16_round", "mlp_param_count", "mlp_unpack", "mlp_init", "mlp_forward",
           "mlp_loss_grad", "adam_step", "warmstart_features", "warmstart_apply",
           "warmstart_targets", "ADAM_B1", "ADAM_B2", "ADAM_EPS"]

ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64. Integer work on the
    float32 bit pattern: add 0x7FFF plus the lowest kept bit, drop the low 16 bits."""
    u = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32)).view(np.uint32)
    u = u.astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (u.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def mlp_param_count(F, Hd, r):
    return F * Hd + Hd + Hd * Hd + Hd + Hd * r + r


def mlp_unpack(params, F, Hd, r):
    p = np.asarray(params, np.float64)
    sizes = [F * Hd, Hd, Hd * Hd, Hd, Hd * r, r]
    out, at = [], 0
    for s in sizes:
        out.append(p[at:at + s])
        at += s
    W1, b1, W2, b2, W3, b3 = out
    return W1.reshape(F, Hd), b1, W2.reshape(Hd, Hd), b2, W3.reshape(Hd, r), b3


def mlp_init(F, Hd, r, seed):
    """He-uniform first two layers, zero last layer (the untrained network is the identity
    correction: W_0 = W_b, H_0 = H_b), zero biases."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (F, Hd)) * np.sqrt(6.0 / F)
    W2 = rng.uniform(-1, 1, (Hd, Hd)) * np.sqrt(6.0 / Hd)
    return np.concatenate([W1.ravel(), np.zeros(Hd), W2.ravel(), np.zeros(Hd),
                           np.zeros(Hd * r), np.zeros(r)])


def mlp_forward(params, X, F, Hd, r, round_weights=True):
    """Rows of X (B x F) through the network; returns Y (B x r) and the activations."""
    W1, b1, W2, b2, W3, b3 = mlp_unpack(params, F, Hd, r)
    if round_weights:
        W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    X = np.asarray(X, np.float64)
    Z1 = X @ W1 + b1
    A1 = np.maximum(Z1, 0.0)
    Z2 = A1 @ W2 + b2
    A2 = np.maximum(Z2, 0.0)
    Y = A2 @ W3 + b3
    return Y, (X, Z1, A1, Z2, A2, W1, W2, W3)


def mlp_loss_grad(params, X, T, F, Hd, r, round_weights=True):
    """L = mean((Y - T)^2) over the B x r outputs and its gradient (chain rule through the two
    ReLU layers; the derivative of relu is taken as 1 where its input is > 0)."""
    Y, (X, Z1, A1, Z2, A2, W1, W2, W3) = mlp_forward(params, X, F, Hd, r, round_weights)
    T = np.asarray(T, np.float64)
    B = X.shape[0]
    E = Y - T
    loss = float(np.mean(E * E))
    G3 = 2.0 * E / (B * r)
    dW3 = A2.T @ G3
    db3 = G3.sum(0)
    G2 = (G3 @ W3.T) * (Z2 > 0)
    dW2 = A1.T @ G2
    db2 = G2.sum(0)
    G1 = (G2 @ W2.T) * (Z1 > 0)
    dW1 = X.T @ G1
    db1 = G1.sum(0)
    grad = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, grad


def adam_step(params, m, v, grad, step, lr, b1=ADAM_B1, b2=ADAM_B2, eps=ADAM_EPS):
    """Adam (Kingma & Ba 2015) with bias correction; step counts from 1."""
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * grad
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return np.asarray(params, np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v


def _part(x, mode):
    if mode == 0:
        return np.abs(x)
    if mode == 1:
        return _pos(x)
    if mode == 2:
        return _neg(x)
    return np.zeros_like(x)


def warmstart_features(QL, Xhat, r):
    """W_b, H_b, hscale, F_w, F_h of the module docstring from the LAPACK SVD of X_hat."""
    QL = np.asarray(QL, np.float64)
    Xhat = np.asarray(Xhat, np.float64)
    m, n = QL.shape[0], Xhat.shape[1]
    U1, s, Vt = np.linalg.svd(Xhat, full_matrices=False)
    U = QL @ U1[:, :r]
    V = Vt[:r].T
    Wb = np.zeros((m, r))
    Hb = np.zeros((r, n))
    hscale = np.zeros(r)
    Fw = np.zeros((m, 3 * r))
    Fh = np.zeros((n, 3 * r))
    for j in range(r):
        x, y = U[:, j], V[:, j]
        if j == 0:
            mode = 0
        else:
            mp = np.linalg.norm(_pos(x)) * np.linalg.norm(_pos(y))
            mn = np.linalg.norm(_neg(x)) * np.linalg.norm(_neg(y))
            mode = (1 if mp > 0 else 3) if mp >= mn else 2
        px, py = _part(x, mode), _part(y, mode)
        nx, ny = np.linalg.norm(px), np.linalg.norm(py)
        if mode != 3 and nx > 0 and ny > 0:
            f2 = s[j] * nx * ny
            Wb[:, j] = px / nx
            Hb[j, :] = f2 * py / ny
            hscale[j] = f2
        sgn = {0: 0.0, 1: 1.0, 2: -1.0, 3: 0.0}[mode]
        Fw[:, j] = np.sqrt(m) * (np.abs(x) if mode == 0 else sgn * x)
        Fh[:, j] = np.sqrt(n) * (np.abs(y) if mode == 0 else sgn * y)
        Fw[:, r + j] = np.sqrt(m) * Wb[:, j]
        Fh[:, r + j] = np.sqrt(n) * (Hb[j, :] / hscale[j] if hscale[j] > 0 else 0.0)
        Fw[:, 2 * r + j] = s[j] / s[0] if s[0] > 0 else 0.0
        Fh[:, 2 * r + j] = s[j] / s[0] if s[0] > 0 else 0.0
    return Wb, Hb, hscale, Fw, Fh


def warmstart_apply(Wb, Hb, hscale, Dw, Dh):
    """Initial factors from the network outputs (module docstring)."""
    m, n = Wb.shape[0], Hb.shape[1]
    W0 = np.maximum(0.0, Wb + np.asarray(Dw, np.float64) / np.sqrt(m))
    H0 = np.maximum(0.0, Hb + np.asarray(hscale)[:, None] * np.asarray(Dh, np.float64).T / np.sqrt(n))
    return W0, H0


def warmstart_targets(Wb, Hb, hscale, Wstar, Hstar):
    """Network targets that map (W_b, H_b) onto a solution (W*, H*): the inverse of
    warmstart_apply where the solution is positive (zero scale components give zero)."""
    m, n = Wb.shape[0], Hb.shape[1]
    Tw = np.sqrt(m) * (np.asarray(Wstar, np.float64) - Wb)
    hs = np.where(np.asarray(hscale) > 0, hscale, 1.0)
    Th = (np.sqrt(n) * (np.asarray(Hstar, np.float64) - Hb) / hs[:, None]).T
    return Tw, Th
