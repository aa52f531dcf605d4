"""Krylov fallback of sgn_solve (Sec. 5, "Solving the saddle point problem":
BiCGSTAB preconditioned by an LDL^T factor of the stabilized matrix).  The
stationary FP64 refinement stalls when the factor is of a matrix far enough
from M; BiCGSTAB, right-preconditioned by the same factor, still reaches the
solution of M.  The oracle is that solution (SuperLU on the CPU)."""
import numpy as np
import pytest

from oracle import equilibrium as EQ
from oracle import system as S
from sgn_inputs import problem_3d

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


@pytest.fixture(scope="module")
def case():
    prob = problem_3d(7, seed=3, p_sigma=0.2)
    x, _ = EQ.newton(prob, prob.p0)
    b = S.blocks(prob, x, prob.p0)
    _, dp, _ = S.sgn_step(b, "kkt")
    # a stabilization of 1% of K's largest diagonal entry: the factor is then
    # of a matrix different enough from M that refinement stalls
    eps = 0.01 * float(np.abs(b.K.diagonal()).max())
    return prob, x, dp, eps


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec_name", ["FP64", "MIXED"])
def test_refinement_stalls_on_a_stabilized_factor(P, case, prec_name):
    prob, x, dp_ref, eps = case
    s = P.SGN.from_problem(prob, stores=P.STORE_FP64 | P.STORE_MIXED)
    s.assemble(x, prob.p0)
    s.factor(getattr(P, prec_name), eps_x=eps, eps_lambda=eps)
    with pytest.raises(P.SGNError) as e:
        s.solve(P.RHS_KKT, method=P.binding.SOLVE_REFINE, max_refine=30)
    assert e.value.code == P.binding.EREFINE
    s.close()


@pytest.mark.parametrize("prec_name,tol", [("FP64", 1e-9), ("MIXED", 1e-8)])
def test_bicgstab_recovers_the_solution(P, case, prec_name, tol):
    """SGN_SOLVE_AUTO: refinement stops contracting, BiCGSTAB takes over from
    its iterate and meets the tolerance; dp equals the oracle's."""
    prob, x, dp_ref, eps = case
    s = P.SGN.from_problem(prob, stores=P.STORE_FP64 | P.STORE_MIXED)
    s.assemble(x, prob.p0)
    s.factor(getattr(P, prec_name), eps_x=eps, eps_lambda=eps)
    _, dp, _, rep = s.solve(P.RHS_KKT)
    assert rep.krylov_iters > 0
    assert rep.residual <= 1e-12
    assert _rel(dp.cpu().numpy(), dp_ref) < tol
    # the factor of M itself afterwards: plain refinement, no Krylov
    s.factor(getattr(P, prec_name))
    _, dp, _, rep = s.solve(P.RHS_KKT)
    assert rep.krylov_iters == 0 and _rel(dp.cpu().numpy(), dp_ref) < tol
    s.close()


def test_bicgstab_from_the_start_and_paper_stabilization(P, case):
    """SGN_SOLVE_BICGSTAB with the FP32 factor of M (whose first solve is
    only FP32-accurate) converges in a few iterations; with the FP64 factor
    the first solve already meets the tolerance and no iteration runs; with
    the paper's stabilization (eps_x = eps_lambda = 1e-6) the default path
    needs no Krylov iterations at all."""
    prob, x, dp_ref, eps = case
    s = P.SGN.from_problem(prob, stores=P.STORE_FP64 | P.STORE_MIXED)
    s.assemble(x, prob.p0)
    s.factor(P.MIXED)
    _, dp, _, rep = s.solve(P.RHS_KKT, method=P.binding.SOLVE_BICGSTAB)
    assert rep.refine_steps == 0 and 1 <= rep.krylov_iters <= 10 and rep.residual <= 1e-12
    assert _rel(dp.cpu().numpy(), dp_ref) < 1e-8
    s.factor(P.FP64)
    _, dp, _, rep = s.solve(P.RHS_KKT, method=P.binding.SOLVE_BICGSTAB)
    assert rep.krylov_iters == 0 and rep.residual <= 1e-12
    assert _rel(dp.cpu().numpy(), dp_ref) < 1e-9
    s.factor(P.FP64, eps_x=1e-6, eps_lambda=1e-6)
    _, dp, _, rep = s.solve(P.RHS_KKT)
    assert rep.krylov_iters == 0 and _rel(dp.cpu().numpy(), dp_ref) < 1e-9
    s.close()
