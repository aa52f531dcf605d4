"""The 80^3-node cube (512,000 nodes, 2,958,234 tets, N = 5,991,834
saddle-point unknowns, the 40^3 cube's total load) in the mixed path: FP32 fronts (tensor-core trailing
updates), FP64 pivots decisions, residuals and refinement.  The oracle cannot
factor this size, so the checks are the properties that hold at any size:
Newton reaches ||c|| <= 1e-10 ||f_ext||, the factorization has the
saddle-point inertia (n_x + n_p, n_x, 0), and refinement drives the FP64
residual of the full system to the round-off floor."""
import numpy as np
import pytest

from sgn_inputs import make_preset

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


def test_kuhn3d_80_mixed_equilibrium_and_step(P):
    prob = make_preset("kuhn3d_80")
    free = torch.cuda.mem_get_info()[0]
    s = P.SGN.from_problem(prob, stores=P.STORE_MIXED | P.STORE_KFACT_MIXED)
    assert s.buf.numel() < free
    x, rep = s.equilibrium(prob.p0, prob.fext, precision=P.MIXED)
    assert rep.converged and rep.residual <= 1e-10, (rep.iters, list(rep.history)[:rep.iters + 1])
    p = torch.as_tensor(prob.p0, device="cuda")
    _, dp, _, frep, srep = s.step(x, p, P.MIXED)
    n_x = prob.n_free * 3
    assert (frep.n_pos, frep.n_neg, frep.n_zero) == (n_x + prob.n_elem, n_x, 0)
    assert frep.tensor_core_updates > 0
    assert srep.residual <= 1e-12, (srep.refine_steps, list(srep.history)[:srep.refine_steps + 1])
    assert bool(torch.isfinite(dp).all()) and float(torch.linalg.norm(dp)) > 0
    s.close()
