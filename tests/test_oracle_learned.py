"""Pins of the learned-warm-start oracle: GELU against its closed form and
finite differences, MLP gradients against finite differences, AdamW's first
step against its closed form, the snapshot basis against orthonormality and
exact reconstruction, the RBF map at a centre."""
import numpy as np
import pytest

from oracle import learned as LR
from sgn_inputs import problem_rbf3d


def test_gelu_values_and_derivative():
    # gelu(0) = 0, gelu(z) -> z for large z, gelu(-z) = gelu(z) - z
    z = np.linspace(-6, 6, 121)
    assert LR.gelu(np.array([0.0]))[0] == 0.0
    np.testing.assert_allclose(LR.gelu(np.array([40.0])), [40.0])
    np.testing.assert_allclose(LR.gelu(-z), LR.gelu(z) - z, atol=1e-14)
    h = 1e-6
    fd = (LR.gelu(z + h) - LR.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(LR.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    params = LR.mlp_init([5, 7, 6, 3], seed=1)
    params = [p + 0.1 * rng.standard_normal(p.shape) for p in params]
    X = rng.standard_normal((4, 5))
    T = rng.standard_normal((4, 3))
    loss, grads = LR.mlp_loss_and_grads(params, X, T)
    h = 1e-6
    for i, P in enumerate(params):
        flat = P.reshape(-1)
        for j in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[j]
            flat[j] = old + h
            lp, _ = LR.mlp_loss_and_grads(params, X, T)
            flat[j] = old - h
            lm, _ = LR.mlp_loss_and_grads(params, X, T)
            flat[j] = old
            fd = (lp - lm) / (2 * h)
            assert abs(grads[i].reshape(-1)[j] - fd) <= 1e-7 * max(1.0, abs(fd)), (i, j)


def test_adamw_first_step_closed_form():
    """At t = 1, m_hat = g and v_hat = g^2, so w -= lr (g / (|g| + eps) + wd w)."""
    w = [np.array([1.0, -2.0, 0.5])]
    g = [np.array([0.3, -1e-3, 2.0])]
    m = [np.zeros(3)]
    v = [np.zeros(3)]
    lr, wd, eps = 0.01, 0.1, 1e-8
    w1, _, _ = LR.adamw_step([w[0].copy()], g, m, v, 1, lr, wd, eps=eps)
    want = w[0] - lr * (g[0] / (np.abs(g[0]) + eps) + wd * w[0])
    np.testing.assert_allclose(w1[0], want, rtol=1e-12)


def test_snapshot_basis_is_orthonormal_and_reconstructs_low_rank_data():
    rng = np.random.default_rng(4)
    base = rng.standard_normal((200, 5))
    coef = rng.standard_normal((5, 40))
    snaps = base @ coef + rng.standard_normal((200, 1))
    mean, U, s = LR.snapshot_basis(snaps, 5)
    np.testing.assert_allclose(U.T @ U, np.eye(5), atol=1e-12)
    rec = mean[:, None] + U @ (U.T @ (snaps - mean[:, None]))
    np.testing.assert_allclose(rec, snaps, atol=1e-10)
    assert np.all(np.diff(s) <= 0)


def test_rbf_map_at_a_centre():
    prob = problem_rbf3d(4)
    Phi = LR.rbf_matrix(prob)
    assert Phi.shape == (prob.n_elem, prob.meta["n_rbf"])
    cent = prob.X[prob.conn].mean(axis=1)
    c = prob.meta["rbf_centers"]
    w = prob.meta["rbf_width"]
    e, k = 3, 5
    np.testing.assert_allclose(Phi[e, k], np.exp(-np.sum((cent[e] - c[k]) ** 2) / (2 * w * w)), rtol=1e-14)
    assert np.all((Phi > 0) & (Phi <= 1))
