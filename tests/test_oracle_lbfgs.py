"""Pins of the oracle's SGN-initialised L-BFGS (oracle/lbfgs.py): the
two-loop recursion against properties fixed by the BFGS update itself, and
the optimisation loop's first step against the dense Gauss-Newton step."""
import numpy as np

from oracle import lbfgs as LB
from oracle import system as S
from oracle import equilibrium as EQ
from sgn_inputs import problem_tiny_2d


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n))
    return a @ a.T + n * np.eye(n)


def test_no_pairs_gives_the_initial_inverse_hessian_step():
    Q = _spd(6, 1)
    g = np.random.default_rng(2).standard_normal(6)
    d = LB.two_loop(g, [], lambda v: np.linalg.solve(Q, v))
    np.testing.assert_allclose(d, -np.linalg.solve(Q, g), rtol=1e-13)


def test_secant_equation_holds_for_the_newest_pair():
    """BFGS makes H_k y_{k-1} = s_{k-1} whatever H_0 is: the two-loop
    recursion applied to y_{k-1} must return -s_{k-1}."""
    rng = np.random.default_rng(3)
    Q = _spd(7, 4)
    pairs = []
    for _ in range(4):
        s = rng.standard_normal(7)
        pairs.append((s, Q @ s))
    d = LB.two_loop(pairs[-1][1], pairs, lambda v: 0.37 * v)
    np.testing.assert_allclose(d, -pairs[-1][0], rtol=1e-11, atol=1e-12)


def test_exact_initial_inverse_is_kept():
    """With H_0 = Q^{-1} and pairs y = Q s of the same quadratic, every BFGS
    update keeps H = Q^{-1}: the direction is -Q^{-1} g for any g (a wrong
    sign, loop order or rho breaks this)."""
    rng = np.random.default_rng(5)
    Q = _spd(8, 6)
    pairs = [(s, Q @ s) for s in rng.standard_normal((5, 8))]
    g = rng.standard_normal(8)
    d = LB.two_loop(g, pairs, lambda v: np.linalg.solve(Q, v))
    np.testing.assert_allclose(d, -np.linalg.solve(Q, g), rtol=1e-10, atol=1e-12)


def test_first_direction_is_the_gauss_newton_step_and_f_decreases():
    prob = problem_tiny_2d()
    x, _ = EQ.newton(prob, prob.p0)
    dp_gn, _, _, _, _ = S.dense_gn(S.blocks(prob, x, prob.p0))
    h0_inv, g = LB.gn_inverse(prob, x, prob.p0)
    np.testing.assert_allclose(LB.two_loop(g, [], h0_inv), dp_gn, rtol=1e-10)
    _, fh, gh = LB.optimize(prob, prob.p0, iters=4, m=3)
    assert all(b <= a for a, b in zip(fh, fh[1:])) and fh[-1] < 0.9 * fh[0]
