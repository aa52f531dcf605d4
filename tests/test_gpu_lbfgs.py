"""SGN-initialised L-BFGS on the GPU (sgn_lbfgs_direction,
sgn_optimize_lbfgs) against the oracle (oracle/lbfgs.py): the two-loop
direction with the Gauss-Newton inverse as H_0, and whole iterations of the
optimiser (equilibria, adjoint gradients, line search)."""
import numpy as np
import pytest

from oracle import equilibrium as EQ
from oracle import lbfgs as LB
from oracle import system as S
from sgn_inputs import problem_2d, problem_tiny_2d

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


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


@pytest.mark.parametrize("m,prec_name,tol", [(0, "FP64", 1e-9), (3, "FP64", 1e-9), (3, "MIXED", 1e-8)])
def test_direction_matches_oracle_two_loop(P, m, prec_name, tol):
    """grid2d_21 at its equilibrium: pairs y = H s from the dense Gauss-Newton
    matrix H (so y.s > 0), g = df/dp; the GPU direction equals the oracle's
    two-loop recursion with H_0^{-1} = H^{-1} (m = 0: the SGN step)."""
    prob = problem_2d()
    x, _ = EQ.newton(prob, prob.p0)
    b = S.blocks(prob, x, prob.p0)
    dp_gn, _, H, g, _ = S.dense_gn(b)
    rng = np.random.default_rng(7)
    Smat = 1e-2 * rng.standard_normal((m, prob.n_elem))
    Ymat = Smat @ H.T if m else np.zeros((0, prob.n_elem))
    h0_inv, g2 = LB.gn_inverse(prob, x, prob.p0)
    want = LB.two_loop(g, [(Smat[i], Ymat[i]) for i in range(m)], h0_inv)
    if m == 0:
        assert _rel(want, dp_gn) < 1e-12
    s = P.SGN.from_problem(prob, stores=P.STORE_FP64 | P.STORE_MIXED)
    s.assemble(x, prob.p0)
    s.factor(getattr(P, prec_name))
    d = s.lbfgs_direction(Smat if m else None, Ymat if m else None, g).cpu().numpy()
    assert _rel(d, want) < tol
    s.close()


def test_objective_value_matches_oracle(P):
    prob = problem_2d()
    x, _ = EQ.newton(prob, prob.p0)
    s = P.SGN.from_problem(prob, stores=P.STORE_KFACT)
    assert abs(s.objective(x, prob.p0) - S.objective(prob, x, prob.p0)) <= 1e-13 * S.objective(prob, x, prob.p0)
    s.close()


def test_optimizer_iterations_match_oracle(P):
    """Three iterations with m = 2 from the design p0 on a small grid (FP64
    factor and FP64 Newton): the same accepted steps, objective values and
    iterates as the oracle's loop, and a monotone decrease."""
    prob = problem_tiny_2d()
    p_ref, fh_ref, gh_ref = LB.optimize(prob, prob.p0, iters=3, m=2)
    s = P.SGN.from_problem(prob, stores=P.STORE_FP64 | P.STORE_KFACT)
    p, x, rep = s.optimize_lbfgs(prob.p0, prob.fext, m=2, max_iter=3, precision=P.FP64, eq_precision=P.FP64)
    assert rep.iters == 3
    fh = list(rep.f)[:4]
    np.testing.assert_allclose(fh, fh_ref, rtol=1e-8)
    assert all(b <= a for a, b in zip(fh, fh[1:]))
    assert _rel(p.cpu().numpy(), p_ref) < 1e-6
    s.close()


def test_mixed_optimizer_follows_the_fp64_one(P):
    """grid2d_21, five iterations with m = 5: FP32 saddle-point fronts with
    FP64 refinement and mixed Newton take the FP64 path's steps (the same
    objective values to 1e-7) and lower f monotonically."""
    prob = problem_2d()
    s = P.SGN.from_problem(prob, stores=P.STORE_FP64 | P.STORE_MIXED | P.STORE_KFACT | P.STORE_KFACT_MIXED)
    _, _, r64 = s.optimize_lbfgs(prob.p0, prob.fext, m=5, max_iter=5, precision=P.FP64, eq_precision=P.FP64)
    _, _, rmx = s.optimize_lbfgs(prob.p0, prob.fext, m=5, max_iter=5, precision=P.MIXED, eq_precision=P.MIXED)
    f64, fmx = list(r64.f)[:6], list(rmx.f)[:6]
    np.testing.assert_allclose(fmx, f64, rtol=1e-7)
    assert all(b <= a for a, b in zip(fmx, fmx[1:])) and fmx[-1] < fmx[0]
    s.close()
