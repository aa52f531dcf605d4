"""Pins of the oracle's assembled system: forward equilibrium, the
sensitivity matrix against finite differences of the equilibrium map
(Eq. dxdp), the total gradient against finite differences of f(x(p), p)
(Eq. totalGradient), Gauss-Newton built by brute force from finite-difference
residual Jacobians (Eq. HGN, Eq. newtonStep), Theorem 1 (sparse == dense),
Theorem 2 (Newton-KKT right-hand side), the saddle-point inertia and the
a-posteriori step error bound."""
import numpy as np
import pytest

from oracle import equilibrium as EQ
from oracle import system as S
from sgn_inputs import problem_2d, problem_tiny_2d, problem_tiny_3d


def _equilibrium(prob, p, x0=None, tol=2e-12):
    # 2e-12 is about the round-off floor of ||c|| / ||f_ext|| on the tiny
    # meshes (the floor grows with the mesh: ~6e-11 on the 21x21 grid)
    x, info = EQ.newton(prob, p, x0=x0, tol=tol, max_iter=60)
    # converged, possibly by stagnating just above tol at the round-off floor
    assert info["converged"] and info["residual"] <= 5 * tol, info
    return x


@pytest.fixture(scope="module", params=["2d", "3d"])
def tiny(request):
    prob = problem_tiny_2d() if request.param == "2d" else problem_tiny_3d()
    p = prob.p0.copy()
    x = _equilibrium(prob, p)
    return prob, p, x


def test_newton_reaches_equilibrium_monotonically():
    prob = problem_2d()
    x, info = EQ.newton(prob, prob.p0)
    assert info["converged"] and info["residual"] <= 1e-10
    # fast local convergence: some Newton step cuts the residual by > 1e3
    h = info["history"]
    assert all(b < a for a, b in zip(h, h[1:]))
    assert min(b / a for a, b in zip(h, h[1:])) < 1e-3


def test_sensitivity_matches_finite_differences(tiny):
    prob, p, x = tiny
    b = S.blocks(prob, x, p)
    Smat = S.sensitivity(b)
    hstep = 1e-4
    fd = np.zeros_like(Smat)
    for e in range(prob.n_elem):
        pp = p.copy(); pp[e] += hstep
        pm = p.copy(); pm[e] -= hstep
        xp = S.free_from_positions(prob, _equilibrium(prob, pp, x))
        xm = S.free_from_positions(prob, _equilibrium(prob, pm, x))
        fd[:, e] = (xp - xm) / (2 * hstep)
    err = np.linalg.norm(Smat - fd) / np.linalg.norm(Smat)
    assert err < 1e-6, err


def test_total_gradient_matches_finite_differences(tiny):
    prob, p, x = tiny
    b = S.blocks(prob, x, p)
    g = S.total_gradient(b)
    hstep = 1e-4
    fd = np.zeros_like(g)
    for e in range(prob.n_elem):
        pp = p.copy(); pp[e] += hstep
        pm = p.copy(); pm[e] -= hstep
        fp_ = S.objective(prob, _equilibrium(prob, pp, x), pp)
        fm_ = S.objective(prob, _equilibrium(prob, pm, x), pm)
        fd[e] = (fp_ - fm_) / (2 * hstep)
    assert np.linalg.norm(g - fd) / np.linalg.norm(g) < 1e-6


def test_gauss_newton_from_residual_jacobians(tiny):
    """Brute force: r(p) = [sqrt(w)(x_t(p) - target); sqrt(alpha) p], J = dr/dp
    by central differences of the equilibrium map, H = J^T J, g = J^T r,
    dp = -H^{-1} g.  Agrees with the SGN step to the FD accuracy."""
    prob, p, x = tiny
    sw = np.sqrt(prob.weight)

    def resid(pv, xguess):
        xe = _equilibrium(prob, pv, xguess)
        return np.concatenate([sw * (xe.reshape(-1)[prob.track_dof] - prob.target),
                               np.sqrt(prob.alpha) * pv])

    r0 = resid(p, x)
    hstep = 1e-4
    J = np.zeros((r0.shape[0], p.shape[0]))
    for e in range(p.shape[0]):
        pp = p.copy(); pp[e] += hstep
        pm = p.copy(); pm[e] -= hstep
        J[:, e] = (resid(pp, x) - resid(pm, x)) / (2 * hstep)
    dp_bf = -np.linalg.solve(J.T @ J, J.T @ r0)
    b = S.blocks(prob, x, p)
    _, dp, _ = S.sgn_step(b, "paper")
    assert np.linalg.norm(dp - dp_bf) / np.linalg.norm(dp_bf) < 1e-5


@pytest.mark.parametrize("which", ["tiny2d", "tiny3d", "grid2d_21"])
def test_theorem1_sparse_equals_dense(which):
    prob = {"tiny2d": problem_tiny_2d, "tiny3d": problem_tiny_3d, "grid2d_21": problem_2d}[which]()
    x = _equilibrium(prob, prob.p0, tol=1e-10)
    b = S.blocks(prob, x, prob.p0)
    dp_d, dx_d, H, g, Sm = S.dense_gn(b)
    for mode in ("paper", "kkt"):
        dx, dp, dl = S.sgn_step(b, mode)
        assert np.linalg.norm(dp - dp_d) / np.linalg.norm(dp_d) < 1e-9
        assert np.linalg.norm(dx - dx_d) / np.linalg.norm(dx_d) < 1e-9


def test_theorem2_multiplier_shift(tiny):
    """KKT right-hand side [-f_x; -f_p; 0] and paper right-hand side
    [0; -df/dp; 0] give the same dp; their dlambda differ by the adjoint
    multipliers -K^{-T} f_x."""
    prob, p, x = tiny
    b = S.blocks(prob, x, p)
    dxk, dpk, dlk = S.sgn_step(b, "kkt")
    dxp, dpp, dlp = S.sgn_step(b, "paper")
    assert np.linalg.norm(dpk - dpp) / np.linalg.norm(dpp) < 1e-10
    lam = S.adjoint(b)
    assert np.linalg.norm(dlk - dlp - lam) / np.linalg.norm(lam) < 1e-9


def test_kkt_inertia(tiny):
    prob, p, x = tiny
    b = S.blocks(prob, x, p)
    n_x, n_p = b.K.shape[0], b.C.shape[0]
    assert S.inertia(S.kkt_matrix(b)) == (n_x + n_p, n_x, 0)


def test_step_error_bound_is_valid(tiny):
    prob, p, x = tiny
    b = S.blocks(prob, x, p)
    _, dp, _ = S.sgn_step(b, "kkt")
    bound0, _ = S.step_error_bound(b, dp)
    assert bound0 < 1e-8 * np.linalg.norm(dp)
    rng = np.random.default_rng(5)
    e = 1e-3 * np.linalg.norm(dp) * rng.standard_normal(dp.shape) / np.sqrt(dp.size)
    bound, _ = S.step_error_bound(b, dp + e)
    assert bound >= np.linalg.norm(e) * (1 - 1e-9)


def test_planted_sign_error_in_cp_is_caught(tiny, monkeypatch):
    """A flipped sign of dc/dp must break the finite-difference pin of S."""
    prob, p, x = tiny
    orig = S.param_jacobian
    monkeypatch.setattr(S, "param_jacobian", lambda *a: -orig(*a))
    with pytest.raises(AssertionError):
        test_sensitivity_matches_finite_differences((prob, p, x))


def test_newton_iterate_is_translation_invariant():
    """The Newton iterate is the displacement, so moving the whole problem
    (rest shape and targets) changes nothing: the same displacements, the
    same residual history, and the 1e-10 tolerance is met although the body
    sits far from the origin (from absolute positions the round-off floor
    there is about 2e-8 ||f_ext||).  The unmoved problem pins the moved one."""
    from sgn_inputs import problem_2d
    # grid spacing 1/16 and an offset of 32: the moved rest shape is exact,
    # so the rest geometry (D_m) is bit for bit the same
    a = problem_2d(17, seed=5)
    b = problem_2d(17, seed=5)
    b.X = b.X + 32.0
    b.target = b.target + 32.0
    xa, ia = EQ.newton(a, a.p0)
    xb, ib = EQ.newton(b, b.p0)
    assert ia["converged"] and ib["converged"]
    assert ia["residual"] <= 1e-10 and ib["residual"] <= 1e-10
    np.testing.assert_array_equal(ia["u"], ib["u"])
    assert ia["history"] == ib["history"]


def _indefinite_problem():
    """tiny2d with its tracked weights made negative on one coordinate each:
    A indefinite, and the reduced Hessian indefinite too."""
    from sgn_inputs import problem_tiny_2d
    prob = problem_tiny_2d()
    w = prob.weight.copy()
    w[::2] = -1e4
    prob.weight = w
    x, _ = EQ.newton(prob, prob.p0)
    return prob, x


def test_inertia_correction_finds_the_first_definite_regularization():
    prob, x = _indefinite_problem()
    b = S.blocks(prob, x, prob.p0)
    S0 = S.sensitivity(b)
    H0 = S0.T @ (b.A @ S0) + b.C.toarray()
    assert np.linalg.eigvalsh(H0).min() < 0  # the unregularized step is not a descent one
    delta, dp, H = S.inertia_corrected(b, delta0=1.0)
    assert delta > 0
    assert np.linalg.eigvalsh(H).min() > 0
    Hprev = S0.T @ ((b.A + (delta / 10.0) * np.eye(b.K.shape[0])) @ S0) + b.C.toarray()
    assert delta == 1.0 or np.linalg.eigvalsh(Hprev).min() <= 0
    # the saddle-point inertia test agrees: (n_x + n_p, n_x, 0) exactly when H(delta) > 0
    n_x, n_p = b.K.shape[0], prob.n_elem
    bd = S.regularized_blocks(b, delta)
    assert S.inertia(S.kkt_matrix(bd)) == (n_x + n_p, n_x, 0)
    assert S.inertia(S.kkt_matrix(b)) != (n_x + n_p, n_x, 0)
    # Theorem 1 at delta: the sparse saddle-point step of M(delta) is the dense one
    _, dps, _ = S.sgn_step(bd, "kkt")
    np.testing.assert_allclose(dps, dp, rtol=1e-9, atol=1e-12 * np.abs(dp).max())
