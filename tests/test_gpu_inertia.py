"""Inertia test with diagonal regularization (sgn_factor_inertia) on the GPU
against the oracle (oracle/system.py inertia_corrected): an objective with
negative tracking weights makes the reduced Hessian indefinite; the
factorization's inertia reveals it, the x diagonal is regularized until the
inertia is (n_x + n_p, n_x, 0), and the step of the regularized system
equals the oracle's dense step at the same delta."""
import numpy as np
import pytest

from oracle import equilibrium as EQ
from oracle import system as S
from sgn_inputs import problem_tiny_2d

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


@pytest.mark.parametrize("prec_name,tol", [("FP64", 1e-9), ("MIXED", 1e-8)])
def test_inertia_corrected_step_matches_oracle(P, prec_name, tol):
    prob = problem_tiny_2d()
    w = prob.weight.copy()
    w[::2] = -1e4
    prob.weight = w
    x, _ = EQ.newton(prob, prob.p0)
    b = S.blocks(prob, x, prob.p0)
    delta_ref, dp_ref, _ = S.inertia_corrected(b, delta0=1.0)
    assert delta_ref > 0
    s = P.SGN.from_problem(prob, stores=P.STORE_FP64 | P.STORE_MIXED)
    s.assemble(x, prob.p0)
    prec = getattr(P, prec_name)
    rep = s.factor(prec)
    n_x, n_p = prob.n_free * 2, prob.n_elem
    assert (rep.n_pos, rep.n_neg, rep.n_zero) != (n_x + n_p, n_x, 0)  # the test sees the indefiniteness
    delta, rep = s.factor_inertia(prec, delta0=1.0)
    assert delta == delta_ref
    assert (rep.n_pos, rep.n_neg, rep.n_zero) == (n_x + n_p, n_x, 0)
    _, dp, _, srep = s.solve(P.RHS_KKT, regularized=True)
    dp = dp.cpu().numpy()
    assert np.linalg.norm(dp - dp_ref) / np.linalg.norm(dp_ref) < tol
    assert srep.residual < 1e-11
    s.close()
