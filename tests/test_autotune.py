"""Host logic of the set-up autotuner (paper_2107_03285_gb300/autotune.py):
candidate enumeration, choice of the fastest, the per-pattern cache.  The
timing function is replaced by a table, so no GPU is needed."""
import json

import numpy as np

from paper_2107_03285_gb300 import autotune as A
from paper_2107_03285_gb300 import binding as B
from sgn_inputs import problem_2d, problem_3d


def _table(leaf, panel):
    # a made-up cost surface with its minimum at leaf 16, panel 32
    return 10.0 + (np.log2(leaf) - 4) ** 2 + (np.log2(panel) - 5) ** 2


def test_candidates_cover_the_grid_and_skip_tiny_leaves():
    c2 = A.candidates(2)
    assert (16, 32) in c2 and (64, 32) in c2
    assert all(p in A.PANELS and l in A.LEAVES for l, p in c2)
    # a leaf front of fewer than half a panel of unknowns is not a candidate
    assert A.candidates(2, panels=(32,), leaves=(2, 4)) == [(4, 32)]


def test_choose_picks_the_fastest_and_breaks_ties_by_order():
    t = {(8, 16): 3.0, (16, 32): 2.0, (32, 64): 2.0}
    assert A.choose(t) == A.Choice(16, 32, 2.0)


def test_tune_measures_once_per_pattern_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    prob = problem_2d(8)
    calls = []

    def fake(P, prob_, precision, leaf, panel, x=None):
        calls.append((leaf, panel))
        return _table(leaf, panel)

    best = A.tune(None, prob, B.MIXED, cache_path=path, measure=fake)
    assert (best.leaf_nodes, best.panel) == (16, 32)
    assert len(calls) == len(A.candidates(2))
    data = json.load(open(path))
    key = A.pattern_key(prob, B.MIXED)
    assert data[key]["panel"] == 32 and data[key]["leaf_nodes"] == 16
    assert len(data[key]["timings"]) == len(calls)
    # cached: no new measurement
    again = A.tune(None, prob, B.MIXED, cache_path=path, measure=fake)
    assert again == best and len(calls) == len(A.candidates(2))
    # force re-measures
    A.tune(None, prob, B.MIXED, cache_path=path, measure=fake, force=True)
    assert len(calls) == 2 * len(A.candidates(2))


def test_pattern_key_separates_meshes_and_precisions():
    a, b = problem_2d(8), problem_2d(9)
    assert A.pattern_key(a, B.MIXED) != A.pattern_key(b, B.MIXED)
    assert A.pattern_key(a, B.MIXED) != A.pattern_key(a, B.FP64)
    # loads and targets do not change the pattern
    c = problem_2d(8, seed=5)
    assert A.pattern_key(a, B.MIXED) == A.pattern_key(c, B.MIXED)
    assert A.pattern_key(problem_3d(3), B.MIXED) != A.pattern_key(a, B.MIXED)


def test_unreadable_cache_is_ignored(tmp_path):
    path = tmp_path / "bad.json"
    path.write_text("{not json")
    assert A.load_cache(str(path)) == {}
    best = A.tune(None, problem_2d(6), B.FP64, cache_path=str(path),
                  measure=lambda *a, **k: 1.0, cands=[(8, 16)])
    assert best == A.Choice(8, 16, 1.0)
