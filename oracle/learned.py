"""Oracle of the learned warm start of the equilibrium solve (FP64 NumPy).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper recomputes the equilibrium x(p) after every parameter update by
Newton's method (Sec. 5, "Computing Equilibrium States"); the warm start
predicts a starting point from the design.  Pieces, each the plain definition:

* RBF design map: p_e = sum_k theta_k exp(-|X_e - c_k|^2 / (2 w^2)) at the
  element centroid X_e.
* Displacement basis: mean snapshot u_bar and the leading left singular
  vectors U of the centred snapshot matrix (numpy SVD), singular values s.
* MLP y = W3 gelu(W2 gelu(W1 x + b1) + b2) + b3 with the exact GELU
  gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2, loss
  L = 1/(2 B) sum_b ||y_b - t_b||^2, gradients by backpropagation.
* AdamW (decoupled weight decay): m = b1 m + (1 - b1) g, v = b2 v + (1 -
  b2) g^2, w -= lr (m_hat / (sqrt(v_hat) + eps) + wd w), hats = bias-corrected.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def rbf_matrix(prob) -> np.ndarray:
    """Phi (n_elem, n_rbf): Phi[e, k] = exp(-|X_e - c_k|^2 / (2 w^2))."""
    centroids = prob.X[prob.conn].mean(axis=1)
    c = prob.meta["rbf_centers"]
    w = prob.meta["rbf_width"]
    d2 = ((centroids[:, None, :] - c[None, :, :]) ** 2).sum(axis=2)
    return np.exp(-d2 / (2.0 * w * w))


def snapshot_basis(snaps: np.ndarray, n_modes: int):
    """snaps (n_dof, n_snap) displacement snapshots -> (mean (n_dof,),
    U (n_dof, n_modes) orthonormal, s (n_modes,)) from the SVD of the
    centred snapshot matrix."""
    mean = snaps.mean(axis=1)
    U, s, _ = np.linalg.svd(snaps - mean[:, None], full_matrices=False)
    return mean, U[:, :n_modes], s[:n_modes]


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def mlp_init(sizes, seed):
    """Weights W_l (out, in) ~ U(-1/sqrt(in), 1/sqrt(in)), biases 0."""
    rng = np.random.default_rng(seed)
    params = []
    for i in range(len(sizes) - 1):
        bound = 1.0 / np.sqrt(sizes[i])
        params.append(rng.uniform(-bound, bound, size=(sizes[i + 1], sizes[i])))
        params.append(np.zeros(sizes[i + 1]))
    return params


def mlp_forward(params, X):
    """X (B, in) -> (Y (B, out), cache); GELU after every layer but the last."""
    n_layers = len(params) // 2
    h = X
    cache = [X]
    for l in range(n_layers):
        W, b = params[2 * l], params[2 * l + 1]
        z = h @ W.T + b
        if l < n_layers - 1:
            cache.append(z)
            h = gelu(z)
            cache.append(h)
        else:
            h = z
    return h, cache


def mlp_loss_and_grads(params, X, T):
    """L = 1/(2B) sum ||Y - T||^2 and dL/dparams (same layout as params)."""
    B = X.shape[0]
    Y, cache = mlp_forward(params, X)
    R = Y - T
    loss = 0.5 * np.sum(R * R) / B
    n_layers = len(params) // 2
    grads = [None] * len(params)
    dz = R / B
    for l in range(n_layers - 1, -1, -1):
        h_in = cache[0] if l == 0 else cache[2 * l]
        grads[2 * l] = dz.T @ h_in
        grads[2 * l + 1] = dz.sum(axis=0)
        if l > 0:
            dh = dz @ params[2 * l]
            z_prev = cache[2 * l - 1]
            dz = dh * gelu_grad(z_prev)
    return loss, grads


def adamw_step(params, grads, m, v, t, lr, wd, b1=0.9, b2=0.999, eps=1e-8):
    """One AdamW step (t counts from 1); updates params, m, v in place."""
    for i in range(len(params)):
        m[i] = b1 * m[i] + (1.0 - b1) * grads[i]
        v[i] = b2 * v[i] + (1.0 - b2) * grads[i] ** 2
        mh = m[i] / (1.0 - b1 ** t)
        vh = v[i] / (1.0 - b2 ** t)
        params[i] = params[i] - lr * (mh / (np.sqrt(vh) + eps) + wd * params[i])
    return params, m, v
