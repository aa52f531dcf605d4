"""Batched form through the C ABI (sgn_batch_setup): many independent
plane-strain instances of uneven size behind one handle, assembled, factored
and solved together (one elimination forest, every level of every instance
batched into the same launches).  Every instance's slice of the batched step
must equal the oracle's step of that instance alone."""
import numpy as np
import pytest

from oracle import equilibrium as EQ
from oracle import system as S
from sgn_inputs import batch2d_instances

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


def _oracle(subs):
    """Oracle equilibria of the instances (joined) and their oracle steps."""
    xs, refs = [], []
    for sub in subs:
        xi, info = EQ.newton(sub, sub.p0)
        assert info["converged"]
        xs.append(xi)
        refs.append(S.sgn_step(S.blocks(sub, xi, sub.p0), "kkt")[1])
    return np.concatenate(xs), refs


def _p(subs):
    return np.concatenate([s.p0 for s in subs])


@pytest.mark.parametrize("prec_name,tol", [("FP64", 1e-9), ("MIXED", 1e-8)])
def test_batched_instances_match_single_instance_oracle(P, prec_name, tol):
    subs = batch2d_instances(12, seed=7, side_lo=5, side_hi=24)
    x, refs = _oracle(subs)
    s = P.SGN.from_batch(subs, stores=P.STORE_FP64 | P.STORE_MIXED)
    no, eo = s.batch_offsets()
    np.testing.assert_array_equal(np.diff(no), [sub.n_nodes for sub in subs])
    prec = getattr(P, prec_name)
    _, dp, _, frep, srep = s.step(x, _p(subs), prec)
    dp = dp.cpu().numpy()
    for i, ref in enumerate(refs):
        got = dp[eo[i]:eo[i + 1]]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol, i
    # per-instance FP64 residuals of the saddle-point solve
    assert np.all(s.batch_residuals(P.binding.BATCH_KKT) < 1e-11)
    # the batch is one saddle-point system: its inertia is the sum of the instances'
    n_x = sum(sub.n_free for sub in subs) * 2
    n_p = sum(sub.n_elem for sub in subs)
    assert (frep.n_pos, frep.n_neg, frep.n_zero) == (n_x + n_p, n_x, 0)
    s.close()


def test_batch_of_256_equilibria_and_steps(P):
    """The full batched workload (256 instances, sides U{10..60}): every
    instance's equilibrium residual is below 1e-10 of its own load (the
    Newton iterate is the displacement, so no instance sits on a round-off
    floor), sampled instances equal the oracle's equilibrium and step, and
    the mixed step agrees with the FP64 GPU step everywhere."""
    subs = batch2d_instances(256, seed=0)
    sample = [0, 77, 255]
    refs = {}
    for i in sample:
        xi, info = EQ.newton(subs[i], subs[i].p0)
        assert info["converged"]
        refs[i] = (xi, S.sgn_step(S.blocks(subs[i], xi, subs[i].p0), "kkt")[1])
    s = P.SGN.from_batch(subs, stores=P.STORE_FP64 | P.STORE_MIXED | P.STORE_KFACT)
    no, eo = s.batch_offsets()
    fext = np.concatenate([sub.fext for sub in subs])
    p = _p(subs)
    xg, rep = s.equilibrium(p, fext)
    assert rep.converged, (rep.iters, rep.residual)
    res = s.batch_residuals(P.binding.BATCH_EQUILIBRIUM)
    assert res.shape == (256,) and np.all(res <= 1e-10), res.max()
    xg = xg.cpu().numpy()
    for i in sample:
        np.testing.assert_allclose(xg[no[i]:no[i + 1]], refs[i][0], rtol=0, atol=1e-9)
    _, dp64, _, _, _ = s.step(xg, p, P.FP64)
    dp64 = dp64.cpu().numpy()
    _, dpm, _, _, srep = s.step(xg, p, P.MIXED)
    dpm = dpm.cpu().numpy()
    assert np.linalg.norm(dpm - dp64) / np.linalg.norm(dp64) < 1e-8
    assert np.all(s.batch_residuals(P.binding.BATCH_KKT) < 1e-11)
    for i in sample:
        ref = refs[i][1]
        got = dp64[eo[i]:eo[i + 1]]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-8, i
    s.close()


def test_graph_step_equals_stepwise_calls(P):
    """sgn_step_graph (assemble + factor + solve + fixed refinement as one
    CUDA-graph launch) gives the stepwise result, call after call, and records
    the per-instance residuals inside the graph."""
    subs = batch2d_instances(12, seed=7, side_lo=5, side_hi=24)
    x, refs = _oracle(subs)
    s = P.SGN.from_batch(subs, stores=P.STORE_MIXED)
    _, eo = s.batch_offsets()
    xd = torch.as_tensor(x, device="cuda")
    pd = torch.as_tensor(_p(subs), device="cuda")
    _, dp_ref, _, _, _ = s.step(xd, pd, P.MIXED)
    dp_ref = dp_ref.clone()
    out = (torch.empty_like(xd), torch.empty_like(pd), torch.empty_like(xd))
    for _ in range(3):
        _, dp, _, res = s.step_graph(xd, pd, P.MIXED, refine_steps=4, out=out)
        assert res < 1e-11
        assert float(torch.linalg.norm(dp - dp_ref) / torch.linalg.norm(dp_ref)) < 1e-10
        assert np.all(s.batch_residuals(P.binding.BATCH_KKT) < 1e-11)
    dpn = out[1].cpu().numpy()
    for i, ref in enumerate(refs):
        assert np.linalg.norm(dpn[eo[i]:eo[i + 1]] - ref) / np.linalg.norm(ref) < 1e-8
    s.close()


def test_autotuned_setup_keeps_parity(P, tmp_path):
    """The autotuner times the graph-captured step for a few (leaf, panel)
    pairs, caches the fastest, and the chosen set-up still matches the oracle
    instance by instance."""
    from paper_2107_03285_gb300 import autotune as A
    subs = batch2d_instances(12, seed=7, side_lo=5, side_hi=24)
    x, refs = _oracle(subs)
    cands = [(8, 16), (16, 32), (32, 32)]
    path = str(tmp_path / "tune.json")
    best = A.tune(P, subs, P.MIXED, cache_path=path, x=x, cands=cands, reps=3, warmup=1)
    assert (best.leaf_nodes, best.panel) in cands and best.ms > 0
    assert A.tune(P, subs, P.MIXED, cache_path=path, x=x, cands=cands) == best
    s = P.SGN.from_batch(subs, stores=P.STORE_MIXED, leaf_nodes=best.leaf_nodes, panel=best.panel)
    _, eo = s.batch_offsets()
    _, dp, _, _, _ = s.step(x, _p(subs), P.MIXED)
    dp = dp.cpu().numpy()
    for i, ref in enumerate(refs):
        assert np.linalg.norm(dp[eo[i]:eo[i + 1]] - ref) / np.linalg.norm(ref) < 1e-8, i
    s.close()


def test_sharded_sub_batches_match_oracle(P):
    """Each rank's share of a batch (cost-balanced partition) is itself a
    batch whose step equals the oracle instance by instance."""
    from paper_2107_03285_gb300 import shard
    subs = batch2d_instances(12, seed=7, side_lo=5, side_hi=24)
    x, refs = _oracle(subs)
    no = np.cumsum([0] + [sub.n_nodes for sub in subs])
    parts = shard.partition(shard.instance_costs([int(round(np.sqrt(sub.n_nodes))) for sub in subs]), 2)
    for part in parts:
        mine = [subs[i] for i in part]
        xs = np.concatenate([x[no[i]:no[i + 1]] for i in part])
        s = P.SGN.from_batch(mine, stores=P.STORE_MIXED)
        _, seo = s.batch_offsets()
        _, dp, _, _, _ = s.step(xs, _p(mine), P.MIXED)
        dp = dp.cpu().numpy()
        for k, i in enumerate(part):
            ref = refs[i]
            assert np.linalg.norm(dp[seo[k]:seo[k + 1]] - ref) / np.linalg.norm(ref) < 1e-8, i
        s.close()
