"""GPU parity of the SGN hot path against the CPU oracle, through the C ABI.

Every comparison feeds the same (x, p) to both sides.  Tolerances:
  * assembled saddle-point entries: 1e-12 relative to the largest entry of
    their block (the CUDA path evaluates the same closed forms in another
    order; FP64 rounding differences stay near 1e-15);
  * FP64 step: dp within 1e-9 relative of dense Gauss-Newton (Theorem 1);
  * mixed step (FP32 fronts + FP64 refinement): dp within 1e-8 relative of
    the FP64 oracle step.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import equilibrium as EQ
from oracle import system as S
from sgn_inputs import problem_2d, problem_3d, problem_tiny_2d, problem_tiny_3d

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def sgnmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_03285_gb300 import build as build_mod
    build_mod.build()
    import paper_2107_03285_gb300 as P
    return P


class Case:
    """An instance at an oracle equilibrium with oracle blocks and steps."""

    def __init__(self, prob, x=None):
        self.prob = prob
        self.p = prob.p0.copy()
        self.x = EQ.newton(prob, self.p)[0] if x is None else x
        self.b = S.blocks(prob, self.x, self.p)
        self.dx_k, self.dp_k, self.dl_k = S.sgn_step(self.b, "kkt")
        self.g = S.total_gradient(self.b)
        g2f = S.free_dof_map(prob)
        self.g2f = g2f

    def free_to_nodes(self, v):
        out = np.zeros(self.prob.n_nodes * self.prob.dim)
        m = self.g2f >= 0
        out[m] = v[self.g2f[m]]
        return out.reshape(self.prob.n_nodes, self.prob.dim)


CASES = {
    "grid2d_21": lambda: problem_2d(),
    "tiny2d": lambda: problem_tiny_2d(),
    "tiny3d": lambda: problem_tiny_3d(),
    "kuhn3d_7": lambda: problem_3d(7, seed=3, p_sigma=0.2),
    "kuhn3d_11": lambda: problem_3d(11, seed=4, p_sigma=0.1),
}
_cache = {}


def case(name):
    if name not in _cache:
        _cache[name] = Case(CASES[name]())
    return _cache[name]


def make(P, c, stores=None, **kw):
    stores = stores if stores is not None else (P.STORE_FP64 | P.STORE_MIXED | P.STORE_KFACT)
    return P.SGN.from_problem(c.prob, stores=stores, **kw)


@pytest.mark.parametrize("name", ["grid2d_21", "tiny3d", "kuhn3d_7"])
def test_assembled_matrix_matches_oracle(sgnmod, name):
    c = case(name)
    s = make(sgnmod, c)
    s.assemble(c.x, c.p)
    rows, cols, vals = s.export_kkt()
    prob = c.prob
    d, nn, ne = prob.dim, prob.n_nodes, prob.n_elem
    n_x = prob.n_free * d
    # map library ids (node*d+a | p | lambda) to the oracle's (free DOF | p | lambda)
    def remap(i):
        out = np.empty_like(i)
        xm = i < nn * d
        pm = (i >= nn * d) & (i < nn * d + ne)
        lm = i >= nn * d + ne
        out[xm] = c.g2f[i[xm]]
        out[pm] = n_x + (i[pm] - nn * d)
        out[lm] = n_x + ne + c.g2f[i[lm] - nn * d - ne]
        return out
    r, q = remap(rows), remap(cols)
    assert np.all(r >= 0) and np.all(q >= 0)
    N = 2 * n_x + ne
    Mg = sp.coo_matrix((vals, (r, q)), shape=(N, N)).tocsr()
    Mo = S.kkt_matrix(c.b).tocsr()
    assert Mg.nnz == Mo.nnz
    diff = (Mg - Mo).tocoo()
    # block-relative error: K, cp and the diagonal blocks have different scales
    Kmax = np.abs(c.b.K).max()
    cpmax = np.abs(c.b.cp).max()
    blk_scale = np.where((diff.row < n_x) | (diff.row >= n_x + ne), Kmax, cpmax)
    blk_scale = np.where(((diff.row >= n_x) & (diff.row < n_x + ne)) | ((diff.col >= n_x) & (diff.col < n_x + ne)),
                         cpmax, blk_scale)
    assert np.max(np.abs(diff.data) / blk_scale, initial=0.0) < 1e-12


@pytest.mark.parametrize("name", ["grid2d_21", "tiny2d", "tiny3d", "kuhn3d_7", "kuhn3d_11"])
def test_fp64_step_matches_oracle(sgnmod, name):
    c = case(name)
    s = make(sgnmod, c)
    dx, dp, dl, frep, srep = s.step(c.x, c.p, sgnmod.FP64)
    dp = dp.cpu().numpy()
    assert _rel(dp, c.dp_k) < 1e-9
    assert _rel(dx.cpu().numpy(), c.free_to_nodes(c.dx_k)) < 1e-9
    assert _rel(dl.cpu().numpy(), c.free_to_nodes(c.dl_k)) < 1e-9
    n_x = c.prob.n_free * c.prob.dim
    assert (frep.n_pos, frep.n_neg, frep.n_zero) == (n_x + c.prob.n_elem, n_x, 0)
    assert srep.residual < 1e-12


def test_fp64_step_equals_dense_gauss_newton(sgnmod):
    """Theorem 1 on the 21x21 plane-strain grid: dp(SGN, GPU) == dp(dense GN)."""
    c = case("grid2d_21")
    dp_dense, dx_dense, H, g, Smat = S.dense_gn(c.b)
    s = make(sgnmod, c)
    _, dp, _, _, _ = s.step(c.x, c.p, sgnmod.FP64)
    assert _rel(dp.cpu().numpy(), dp_dense) < 1e-9


def test_paper_rhs_and_multiplier_shift(sgnmod):
    """Eq. sparseSystemGN's right-hand side [0; -g; 0] gives the same dp as
    the KKT form; dlambda shifts by the adjoint multipliers (Theorem 2)."""
    c = case("kuhn3d_7")
    s = make(sgnmod, c)
    s.assemble(c.x, c.p)
    s.factor(sgnmod.FP64)
    dxk, dpk, dlk, _ = s.solve(sgnmod.RHS_KKT)
    dxp, dpp, dlp, _ = s.solve(sgnmod.RHS_PAPER, g=c.g)
    assert _rel(dpp.cpu().numpy(), dpk.cpu().numpy()) < 1e-10
    lam = c.free_to_nodes(S.adjoint(c.b))
    assert _rel((dlk - dlp).cpu().numpy(), lam) < 1e-9


@pytest.mark.parametrize("panel,leaf", [(8, 4), (16, 64), (32, 8)])
def test_panel_and_leaf_sizes(sgnmod, panel, leaf):
    c = case("kuhn3d_7")
    s = make(sgnmod, c, panel=panel, leaf_nodes=leaf)
    _, dp, _, frep, _ = s.step(c.x, c.p, sgnmod.FP64)
    assert _rel(dp.cpu().numpy(), c.dp_k) < 1e-9
    n_x = c.prob.n_free * c.prob.dim
    assert (frep.n_pos, frep.n_neg) == (n_x + c.prob.n_elem, n_x)


@pytest.mark.parametrize("name", ["grid2d_21", "kuhn3d_7", "kuhn3d_11"])
def test_mixed_step_matches_fp64_oracle(sgnmod, name):
    c = case(name)
    s = make(sgnmod, c)
    _, dp, _, frep, srep = s.step(c.x, c.p, sgnmod.MIXED)
    assert _rel(dp.cpu().numpy(), c.dp_k) < 1e-8
    assert srep.refine_steps >= 1
    if name == "kuhn3d_11":
        # fronts larger than one 128-row tile take the tcgen05 trailing update
        assert frep.tensor_core_updates > 0


@pytest.mark.parametrize("name", ["grid2d_21", "kuhn3d_7"])
def test_equilibrium_matches_oracle(sgnmod, name):
    c = case(name)
    s = make(sgnmod, c)
    x, rep = s.equilibrium(c.p, c.prob.fext)
    assert rep.converged and rep.residual <= 1e-10
    assert _rel(x.cpu().numpy(), c.x) < 1e-9


@pytest.mark.parametrize("name", ["grid2d_21", "kuhn3d_11"])
def test_mixed_equilibrium_matches_oracle(sgnmod, name):
    """Newton with FP32 K fronts (tensor-core trailing updates on kuhn3d_11)
    and FP64-refined directions reaches the FP64 equilibrium."""
    c = case(name)
    s = make(sgnmod, c, stores=sgnmod.STORE_KFACT | sgnmod.STORE_KFACT_MIXED)
    x64, rep64 = s.equilibrium(c.p, c.prob.fext)
    x, rep = s.equilibrium(c.p, c.prob.fext, precision=sgnmod.MIXED)
    assert rep.converged and rep.residual <= 1e-10
    assert rep.iters <= rep64.iters + 1
    assert _rel(x.cpu().numpy(), c.x) < 1e-9


def test_mixed_equilibrium_needs_its_store(sgnmod):
    c = case("kuhn3d_7")
    s = make(sgnmod, c, stores=sgnmod.STORE_KFACT)
    with pytest.raises(sgnmod.SGNError) as e:
        s.equilibrium(c.p, c.prob.fext, precision=sgnmod.MIXED)
    assert e.value.code == 8  # ESTATE


def test_gradient_matches_oracle(sgnmod):
    c = case("kuhn3d_7")
    s = make(sgnmod, c)
    s.assemble(c.x, c.p)
    s.factor_k()
    g = s.gradient().cpu().numpy()
    assert _rel(g, c.g) < 1e-9


def test_step_host_equals_device_path(sgnmod):
    c = case("kuhn3d_7")
    s = make(sgnmod, c)
    dxh, dph, dlh, rep = s.step_host(c.x, c.p, sgnmod.FP64)
    _, dp, _, _, _ = s.step(c.x, c.p, sgnmod.FP64)
    assert _rel(dph, dp.cpu().numpy()) < 1e-13
    assert _rel(dph, c.dp_k) < 1e-9


def test_inverted_element_is_reported(sgnmod):
    c = case("tiny2d")
    s = make(sgnmod, c)
    x = c.x.copy()
    e = 0
    a, b = c.prob.conn[e, 1], c.prob.conn[e, 2]
    x[[a, b]] = x[[b, a]]  # swapping two vertices flips det F
    s.assemble(x, c.p)
    with pytest.raises(sgnmod.SGNError) as ei:
        s.factor(sgnmod.FP64, report=True)
    assert ei.value.code == 4  # SGN_EINVERTED


def test_bounded_wait_reports_timeout_and_context_stays_usable(sgnmod):
    """A substitution wait on a block value nothing publishes gives up after
    its bound (about a second), the host reads SGN_ETIMEOUT, and the same
    handle then still takes a correct step: the failure is reported, the
    GPU context is not lost."""
    import time
    c = case("kuhn3d_7")
    s = make(sgnmod, c)
    t0 = time.perf_counter()
    code = s.lib.sgn_selftest_wait_timeout(s.h)
    waited = time.perf_counter() - t0
    assert code == 10  # SGN_ETIMEOUT
    assert 0.1 < waited < 30.0
    _, dp, _, _, _ = s.step(c.x, c.p, sgnmod.MIXED)
    assert _rel(dp.cpu().numpy(), c.dp_k) < 1e-8


@pytest.mark.parametrize("ctas", [1, 3])
def test_tensor_core_update_ctas_loop_over_tiles(sgnmod, ctas):
    """Capping the tensor-core update at a few CTAs makes every CTA walk
    several 128 x 128 tiles of its front, alternating its two TMEM
    accumulators (the persistent loop's buffer hand-off); the step still
    matches the FP64 oracle."""
    c = case("kuhn3d_11")
    s = make(sgnmod, c, update_ctas=ctas)
    _, dp, _, frep, srep = s.step(c.x, c.p, sgnmod.MIXED)
    assert frep.tensor_core_updates > 0
    assert _rel(dp.cpu().numpy(), c.dp_k) < 1e-8
    n_x = c.prob.n_free * c.prob.dim
    assert (frep.n_pos, frep.n_neg, frep.n_zero) == (n_x + c.prob.n_elem, n_x, 0)


def test_mixed_step_error_certificate_kuhn3d_24(sgnmod):
    """A posteriori bound on the mixed GPU step of a 24^3-node cube (N =
    192,490), where dense Gauss-Newton is out of reach: H >= alpha I gives
    ||dp - dp*|| <= ||H dp + g|| / alpha, with H dp and g applied by the
    oracle through two sparse K solves (SuperLU on the CPU).  At this size
    the root front has 27 blocks of 128 columns in each substitution chain
    and every tensor-core CTA loops over several tiles."""
    prob = problem_3d(24, seed=2, p_sigma=0.1)
    s = sgnmod.SGN.from_problem(prob, stores=sgnmod.STORE_MIXED | sgnmod.STORE_KFACT_MIXED)
    x, rep = s.equilibrium(prob.p0, prob.fext, precision=sgnmod.MIXED)
    assert rep.converged and rep.residual <= 1e-10
    x = x.cpu().numpy()
    _, dp, _, frep, srep = s.step(x, prob.p0, sgnmod.MIXED)
    dp = dp.cpu().numpy()
    b = S.blocks(prob, x, prob.p0)
    bound, _ = S.step_error_bound(b, dp)
    assert bound <= 1e-8 * np.linalg.norm(dp), bound / np.linalg.norm(dp)
    n_x = prob.n_free * prob.dim
    assert (frep.n_pos, frep.n_neg, frep.n_zero) == (n_x + prob.n_elem, n_x, 0)


def test_equilibrium_is_translation_invariant(sgnmod):
    """The Newton iterate is the displacement: the same problem moved by 32
    (grid spacing 1/16, so the moved rest shape is exact) takes the same
    iterations to the same residual, below 1e-10, and the same
    displacements."""
    a = problem_2d(17, seed=5)
    b = problem_2d(17, seed=5)
    b.X = b.X + 32.0
    b.target = b.target + 32.0
    out = []
    for prob in (a, b):
        s = sgnmod.SGN.from_problem(prob, stores=sgnmod.STORE_KFACT)
        x, rep = s.equilibrium(prob.p0, prob.fext)
        assert rep.converged and rep.residual <= 1e-10
        out.append(((x.cpu().numpy() - prob.X), list(rep.history)[:rep.iters + 1]))
        s.close()
    assert out[0][1] == out[1][1]
    np.testing.assert_allclose(out[0][0], out[1][0], rtol=0, atol=1e-13)
