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


class _OneTet:
    """A single tetrahedron built so that its centroid is known exactly:
    vertices 0, e_x, e_y, e_z give the centroid (1/4, 1/4, 1/4) (the mean of
    only three of them would be (1/3, 1/3, 0) or similar)."""

    def __init__(self, centers, width):
        self.X = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
        self.conn = np.array([[0, 1, 2, 3]], dtype=np.int32)
        self.meta = {"rbf_centers": np.asarray(centers, dtype=np.float64), "rbf_width": width}


def test_rbf_map_closed_form_values():
    """Phi = exp(-r^2 / (2 w^2)) at the centroid: 1 exactly on a centre,
    exp(-1/2) one width away, exp(-2) two widths away, exp(-9/2) three widths
    away along a diagonal.  A wrong centroid or a width convention without the
    factor 2 fails these."""
    w = 0.15
    g = np.array([0.25, 0.25, 0.25])
    diag = np.array([1.0, 1.0, 1.0]) / np.sqrt(3.0)
    centers = [g, g + [w, 0.0, 0.0], g + [0.0, -2.0 * w, 0.0], g + 3.0 * w * diag]
    Phi = LR.rbf_matrix(_OneTet(centers, w))
    assert Phi.shape == (1, 4)
    assert Phi[0, 0] == 1.0
    np.testing.assert_allclose(Phi[0, 1:], [np.exp(-0.5), np.exp(-2.0), np.exp(-4.5)], rtol=1e-13)


def test_adamw_later_steps_closed_form():
    """Steps 2 and 3 with changing gradients, the bias-corrected moments
    written out by hand for b1 = 0.9, b2 = 0.999:
      t = 2: m_hat = (0.09 g1 + 0.1 g2) / 0.19,
             v_hat = (0.000999 g1^2 + 0.001 g2^2) / 0.001999;
      t = 3: m_hat = (0.081 g1 + 0.09 g2 + 0.1 g3) / 0.271,
             v_hat = (0.000998001 g1^2 + 0.000999 g2^2 + 0.001 g3^2) / 0.002997001.
    A wrong exponent in a bias correction (1 - b^(t-1), 1 - b^(t+1)) or a
    missing correction of v fails them (the corrections cancel at t = 1)."""
    lr, wd, eps = 0.01, 0.1, 1e-8
    g1, g2, g3 = np.array([0.3, -1.0, 2.0]), np.array([-0.5, 0.2, 1.0]), np.array([0.1, 0.7, -3.0])
    w = [np.array([1.0, -2.0, 0.5])]
    m, v = [np.zeros(3)], [np.zeros(3)]
    w1, m, v = LR.adamw_step([w[0].copy()], [g1], m, v, 1, lr, wd, eps=eps)
    w1c = w1[0].copy()
    w2, m, v = LR.adamw_step([w1c.copy()], [g2], m, v, 2, lr, wd, eps=eps)
    mh2 = (0.09 * g1 + 0.1 * g2) / 0.19
    vh2 = (0.000999 * g1 ** 2 + 0.001 * g2 ** 2) / 0.001999
    want2 = w1c - lr * (mh2 / (np.sqrt(vh2) + eps) + wd * w1c)
    np.testing.assert_allclose(w2[0], want2, rtol=1e-12)
    w2c = w2[0].copy()
    w3, m, v = LR.adamw_step([w2c.copy()], [g3], m, v, 3, lr, wd, eps=eps)
    mh3 = (0.081 * g1 + 0.09 * g2 + 0.1 * g3) / 0.271
    vh3 = (0.000998001 * g1 ** 2 + 0.000999 * g2 ** 2 + 0.001 * g3 ** 2) / 0.002997001
    want3 = w2c - lr * (mh3 / (np.sqrt(vh3) + eps) + wd * w2c)
    np.testing.assert_allclose(w3[0], want3, rtol=1e-12)
