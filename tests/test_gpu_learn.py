"""Learned warm start of the equilibrium solve on the GPU (include/sgn_learn.h):
the RBF design map, the randomised-SVD snapshot basis, the BF16 MLP's loss and
gradients and the AdamW step against the FP64 oracle (oracle/learned.py), and
a trained network's gain over starting Newton from the rest shape."""
import numpy as np
import pytest

from oracle import equilibrium as EQ
from oracle import learned as LR
from sgn_inputs import draw_thetas, problem_rbf3d

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_03285_gb300 import build as build_mod
    build_mod.build()
    import paper_2107_03285_gb300 as P
    return P


def _bf16(a):
    """Round float32 values to the nearest BF16 (ties to even), kept as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _small(P, n_modes=8, hidden=32, batch=16, max_snap=64):
    prob = problem_rbf3d(4)
    s = P.SGN.from_problem(prob, stores=P.STORE_KFACT)
    ws = P.WarmStart(s, prob.meta["rbf_centers"], prob.meta["rbf_width"], n_modes=n_modes, hidden=hidden,
                     max_snap=max_snap, batch=batch)
    return prob, s, ws


def test_rbf_design_map_matches_oracle(P):
    prob, s, ws = _small(P)
    Phi = LR.rbf_matrix(prob)
    for th in draw_thetas(prob, 3, seed=5):
        p = ws.rbf_params(th).cpu().numpy()
        np.testing.assert_allclose(p, Phi @ th, rtol=1e-12, atol=1e-14)
    ws.close()
    s.close()


@pytest.mark.parametrize("hidden,batch", [(32, 16), (96, 67)])
def test_mlp_loss_and_gradients_match_oracle(P, hidden, batch):
    """BF16 operands, FP32 accumulation against the FP64 oracle on the same
    (BF16-representable) weights and inputs: the remaining difference is the
    BF16 rounding of the hidden activations, about 2^-9 relative per entry."""
    prob, s, ws = _small(P, hidden=hidden, batch=batch, max_snap=max(64, batch))
    rng = np.random.default_rng(2)
    params = LR.mlp_init([ws.n_rbf, hidden, hidden, ws.n_modes], seed=3)
    params = [p + 0.05 * rng.standard_normal(p.shape) for p in params]
    params = [(_bf16(p) if p.ndim == 2 else p.astype(np.float32)).astype(np.float64) for p in params]
    ws.set_params(np.concatenate([p.ravel() for p in params]).astype(np.float32))
    X = _bf16(rng.standard_normal((batch, ws.n_rbf))).astype(np.float64)
    T = rng.standard_normal((batch, ws.n_modes)).astype(np.float32).astype(np.float64)
    loss, g = ws.grads(X, T)
    loss_ref, g_ref = LR.mlp_loss_and_grads(params, X, T)
    assert abs(loss - loss_ref) <= 1e-2 * loss_ref
    for name, got, ref in zip(["W1", "b1", "W2", "b2", "W3", "b3"], ws.split(g), g_ref):
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 1.5e-2, (name, err)
    ws.close()
    s.close()


def test_adamw_steps_match_oracle(P):
    prob, s, ws = _small(P)
    rng = np.random.default_rng(4)
    p0 = rng.standard_normal(ws.n_params).astype(np.float32)
    ws.set_params(p0)
    w, m, v = [p0.astype(np.float64)], [np.zeros(ws.n_params)], [np.zeros(ws.n_params)]
    for t in (1, 2, 3):
        g = (rng.standard_normal(ws.n_params) * 10.0 ** rng.uniform(-3, 1, ws.n_params)).astype(np.float32)
        ws.apply(g, lr=1e-2, weight_decay=0.1)
        w, m, v = LR.adamw_step(w, [g.astype(np.float64)], m, v, t, 1e-2, 0.1)
    np.testing.assert_allclose(ws.params(), w[0], rtol=1e-5, atol=1e-6)
    ws.close()
    s.close()


@pytest.mark.parametrize("n_snap", [60, 20])
def test_snapshot_basis_matches_oracle_svd(P, n_snap):
    """Snapshots with a geometric spectrum (rank 50; rank-deficient when
    n_snap = 20): mean, orthonormality, the leading 8-mode subspace and the
    singular values against numpy's SVD of the centred matrix."""
    prob, s, ws = _small(P, n_modes=8, max_snap=64)
    nd = prob.n_nodes * 3
    rng = np.random.default_rng(6)
    Qb, _ = np.linalg.qr(rng.standard_normal((nd, 50)))
    sig = 0.6 ** np.arange(50)
    snaps = (rng.standard_normal(nd)[:, None] + Qb @ (sig[:, None] * rng.standard_normal((50, n_snap)))).T
    sigma = ws.fit_basis(snaps.reshape(n_snap, prob.n_nodes, 3), seed=9)
    mean, U = ws.basis()
    mean_ref, U_ref, s_ref = LR.snapshot_basis(snaps.T, 8)
    np.testing.assert_allclose(mean, mean_ref, rtol=0, atol=1e-13)
    np.testing.assert_allclose(U.T @ U, np.eye(8), atol=1e-12)
    np.testing.assert_allclose(sigma, s_ref, rtol=1e-9)
    proj = U @ U.T - U_ref @ U_ref.T
    assert np.linalg.norm(proj, 2) < 1e-8
    ws.close()
    s.close()


@pytest.fixture(scope="module")
def trained(P):
    """rbf3d on an 8-cell cube (729 nodes): 192 GPU equilibria at theta ~
    N(0, 0.3^2) as snapshots, a 32-mode basis and a 64-128-128-32 MLP."""
    prob = problem_rbf3d(8)
    s = P.SGN.from_problem(prob, stores=P.STORE_KFACT)
    ws = P.WarmStart(s, prob.meta["rbf_centers"], prob.meta["rbf_width"], n_modes=32, hidden=128, max_snap=192,
                     batch=32)
    thetas = draw_thetas(prob, 192 + 8, seed=11)
    X = torch.as_tensor(prob.X, device="cuda")
    snaps, cold = [], []
    for th in thetas[:192]:
        x, rep = s.equilibrium(ws.rbf_params(th), prob.fext)
        assert rep.converged
        snaps.append(x - X)
    snaps = torch.stack(snaps)
    ws.fit_basis(snaps, seed=1)
    loss = ws.train(thetas[:192], snaps, steps=3000, lr=2e-3, weight_decay=1e-5, seed=2)
    yield prob, s, ws, thetas[192:], loss
    ws.close()
    s.close()


def test_training_fits_the_snapshots(trained):
    _, _, _, _, loss = trained
    # normalised mean squared error (1 = predicting the mean snapshot)
    assert loss < 0.05, loss


def test_warm_start_saves_newton_iterations(P, trained):
    prob, s, ws, test_thetas, _ = trained
    it_cold, it_warm, r0_warm = [], [], []
    for th in test_thetas:
        xc, rc = s.equilibrium(ws.rbf_params(th), prob.fext)
        xw, rw, used = ws.equilibrium(th, prob.fext)
        assert rc.converged and rw.converged
        assert used
        assert rw.residual < 1e-10
        np.testing.assert_allclose(xw.cpu().numpy(), xc.cpu().numpy(), rtol=0, atol=1e-9)
        it_cold.append(rc.iters)
        it_warm.append(rw.iters)
        r0_warm.append(rw.initial_residual)
    # the rest shape starts at ||c|| / ||f_ext|| = 1.  The force residual weighs
    # the displacement error by the stiffness, so even the exact projection of
    # the equilibrium on 32 modes starts near 0.17 on this mesh; what the
    # prediction buys is about one Newton iteration (4 from rest, 3 warm)
    assert max(r0_warm) < 0.5, r0_warm
    assert np.mean(it_warm) <= np.mean(it_cold) - 0.75, (it_cold, it_warm)


def test_warm_equilibrium_matches_oracle_and_falls_back_to_previous_iterate(P, trained):
    prob, s, ws, test_thetas, _ = trained
    th = test_thetas[0]
    x, rep, used = ws.equilibrium(th, prob.fext)
    x_ref, info = EQ.newton(prob, LR.rbf_matrix(prob) @ th)
    assert info["converged"]
    np.testing.assert_allclose(x.cpu().numpy(), x_ref, rtol=0, atol=1e-8)
    # the previous iterate already is the equilibrium: it wins, Newton stops at once
    x2, rep2, used2 = ws.equilibrium(th, prob.fext, x_prev=x)
    assert not used2
    assert rep2.iters == 0
    np.testing.assert_allclose(x2.cpu().numpy(), x.cpu().numpy(), rtol=0, atol=0)
