"""Batched form: many independent plane-strain instances of uneven size in one
disjoint mesh, assembled, factored and solved together (one elimination
forest, every level of every instance batched into the same launches).
Every instance's slice of the batched step must equal the oracle's step of
that instance alone."""
import numpy as np
import pytest

from oracle import equilibrium as EQ
from oracle import system as S
from sgn_inputs import problem_2d, problem_batch2d

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


def _instances(batch):
    """Rebuild every instance exactly as problem_batch2d drew it."""
    rng = np.random.default_rng(batch.meta["seed"])
    sides = rng.integers(batch.meta["side_lo"], batch.meta["side_hi"] + 1, size=len(batch.meta["sides"]))
    out = []
    for n in sides:
        shift = (0.0, -0.05) + rng.normal(0.0, batch.meta["shift_sigma"], size=2)
        out.append(problem_2d(int(n), seed=int(rng.integers(0, 2**31 - 1)), shift=tuple(shift),
                              p_sigma=batch.meta["p_sigma"]))
    return out


def _batch_state(batch, subs):
    """Oracle equilibria of the instances, placed into the batch mesh."""
    x = batch.X.copy()
    no = batch.meta["node_offsets"]
    refs = []
    for i, sub in enumerate(subs):
        xi, info = EQ.newton(sub, sub.p0)
        assert info["converged"]
        x[no[i]:no[i + 1]] = xi + batch.meta["origins"][i]
        b = S.blocks(sub, xi, sub.p0)
        refs.append(S.sgn_step(b, "kkt")[1])
    return x, refs


@pytest.mark.parametrize("prec_name,tol", [("FP64", 1e-9), ("MIXED", 1e-8)])
def test_batched_instances_match_single_instance_oracle(P, prec_name, tol):
    batch = problem_batch2d(12, seed=7, side_lo=5, side_hi=24)
    subs = _instances(batch)
    assert [s.n_nodes for s in subs] == list(np.diff(batch.meta["node_offsets"]))
    x, refs = _batch_state(batch, subs)
    s = P.SGN.from_problem(batch, stores=P.STORE_FP64 | P.STORE_MIXED)
    prec = getattr(P, prec_name)
    _, dp, _, frep, srep = s.step(x, batch.p0, prec)
    dp = dp.cpu().numpy()
    eo = batch.meta["elem_offsets"]
    for i, ref in enumerate(refs):
        got = dp[eo[i]:eo[i + 1]]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol, i
    # the batch is one saddle-point system: its inertia is the sum of the instances'
    n_x = batch.n_free * 2
    assert (frep.n_pos, frep.n_neg, frep.n_zero) == (n_x + batch.n_elem, n_x, 0)
    s.close()


def test_batch_of_256_runs_and_samples_match_oracle(P):
    """The full batched workload (256 instances, sides U{10..60}): the mixed
    step agrees with the FP64 GPU step everywhere, and sampled instances agree
    with the oracle."""
    batch = problem_batch2d(256, seed=0)
    subs = _instances(batch)
    no, eo = batch.meta["node_offsets"], batch.meta["elem_offsets"]
    x = batch.X.copy()
    sample = [0, 77, 255]
    refs = {}
    for i in sample:
        sub = subs[i]
        xi, info = EQ.newton(sub, sub.p0)
        assert info["converged"]
        refs[i] = (xi, S.sgn_step(S.blocks(sub, xi, sub.p0), "kkt")[1])
    s = P.SGN.from_problem(batch, stores=P.STORE_FP64 | P.STORE_MIXED | P.STORE_KFACT)
    xg, rep = s.equilibrium(batch.p0, batch.fext)
    assert rep.converged, (rep.iters, rep.residual)
    xg = xg.cpu().numpy()
    for i in sample:
        # GPU equilibrium of the batch == oracle equilibrium of the instance
        xi, _ = refs[i]
        np.testing.assert_allclose(xg[no[i]:no[i + 1]] - batch.meta["origins"][i], xi, rtol=0, atol=1e-8)
    _, dp64, _, _, _ = s.step(xg, batch.p0, P.FP64)
    dp64 = dp64.cpu().numpy()
    _, dpm, _, _, srep = s.step(xg, batch.p0, P.MIXED)
    dpm = dpm.cpu().numpy()
    assert np.linalg.norm(dpm - dp64) / np.linalg.norm(dp64) < 1e-8
    for i in sample:
        ref = refs[i][1]
        got = dp64[eo[i]:eo[i + 1]]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-8, i
    s.close()


def test_graph_step_equals_stepwise_calls(P):
    """sgn_step_graph (assemble + factor + solve + fixed refinement as one
    CUDA-graph launch) gives the stepwise result, call after call."""
    batch = problem_batch2d(12, seed=7, side_lo=5, side_hi=24)
    subs = _instances(batch)
    x, refs = _batch_state(batch, subs)
    s = P.SGN.from_problem(batch, stores=P.STORE_MIXED)
    xd = torch.as_tensor(x, device="cuda")
    pd = torch.as_tensor(batch.p0, device="cuda")
    _, dp_ref, _, _, _ = s.step(xd, pd, P.MIXED)
    dp_ref = dp_ref.clone()
    out = (torch.empty_like(xd), torch.empty_like(pd), torch.empty_like(xd))
    for _ in range(3):
        _, dp, _, res = s.step_graph(xd, pd, P.MIXED, refine_steps=4, out=out)
        assert res < 1e-11
        assert float(torch.linalg.norm(dp - dp_ref) / torch.linalg.norm(dp_ref)) < 1e-10
    eo = batch.meta["elem_offsets"]
    dpn = out[1].cpu().numpy()
    for i, ref in enumerate(refs):
        assert np.linalg.norm(dpn[eo[i]:eo[i + 1]] - ref) / np.linalg.norm(ref) < 1e-8
    s.close()


def test_autotuned_setup_keeps_parity(P, tmp_path):
    """The autotuner times the graph-captured step for a few (leaf, panel)
    pairs, caches the fastest, and the chosen set-up still matches the oracle
    instance by instance."""
    from paper_2107_03285_gb300 import autotune as A
    batch = problem_batch2d(12, seed=7, side_lo=5, side_hi=24)
    subs = _instances(batch)
    x, refs = _batch_state(batch, subs)
    cands = [(8, 16), (16, 32), (32, 32)]
    path = str(tmp_path / "tune.json")
    best = A.tune(P, batch, P.MIXED, cache_path=path, x=x, cands=cands, reps=3, warmup=1)
    assert (best.leaf_nodes, best.panel) in cands and best.ms > 0
    assert A.tune(P, batch, P.MIXED, cache_path=path, x=x, cands=cands) == best
    s = P.SGN.from_problem(batch, stores=P.STORE_MIXED, leaf_nodes=best.leaf_nodes, panel=best.panel)
    _, dp, _, _, _ = s.step(x, batch.p0, P.MIXED)
    dp = dp.cpu().numpy()
    eo = batch.meta["elem_offsets"]
    for i, ref in enumerate(refs):
        assert np.linalg.norm(dp[eo[i]:eo[i + 1]] - ref) / np.linalg.norm(ref) < 1e-8, i
    s.close()


def test_sharded_sub_batches_match_oracle(P):
    """Each rank's share of a batch (cost-balanced partition) is itself a
    batch whose step equals the oracle instance by instance."""
    from paper_2107_03285_gb300 import shard
    from sgn_inputs import select_instances
    batch = problem_batch2d(12, seed=7, side_lo=5, side_hi=24)
    subs = _instances(batch)
    x, refs = _batch_state(batch, subs)
    parts = shard.partition(shard.instance_costs(batch.meta["sides"]), 2)
    no = batch.meta["node_offsets"]
    for part in parts:
        sb = select_instances(batch, part)
        xs = np.concatenate([x[no[i]:no[i + 1]] for i in part])
        s = P.SGN.from_problem(sb, stores=P.STORE_MIXED)
        _, dp, _, _, _ = s.step(xs, sb.p0, P.MIXED)
        dp = dp.cpu().numpy()
        seo = sb.meta["elem_offsets"]
        for k, i in enumerate(part):
            ref = refs[i]
            assert np.linalg.norm(dp[seo[k]:seo[k + 1]] - ref) / np.linalg.norm(ref) < 1e-8, i
        s.close()
