"""Autotuner for the set-up options that shape the fronts and their schedule.

Two options of ``sgn_setup`` decide the tile structure of the factorization:
``panel`` (the pivot panel width: the column tile of the Bunch-Kaufman /
TRSM kernels and the K-chunk the trailing tensor-core update consumes per
panel) and ``leaf_nodes`` (where nested dissection stops: the size of the
leaf fronts, hence how many fronts each level batches into one launch and how
deep the level schedule is).  The best pair depends on the mesh: thousands of
small 2D fronts favour narrow panels and small leaves, large 3D separators
favour wide panels.

``tune`` times one graph-captured step (``sgn_step_graph``: assemble, factor,
solve and refinement in one CUDA-graph launch) for every candidate pair on
the caller's mesh and keeps the fastest.  Results are cached per mesh pattern
(a hash of the connectivity, fixed nodes, dimension and precision) in a JSON
file, so a pattern is tuned once.  Timing uses CUDA events on the step's
stream after warm-up launches.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass

import numpy as np

from . import binding as B

PANELS = (16, 32)
LEAVES = (8, 16, 32, 64)
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "sgn_autotune.json")
# tuned choices for the standard workloads, shipped with the package
SHIPPED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def lookup(prob, precision, paths=(SHIPPED, DEFAULT_CACHE)):
    """(leaf_nodes, panel) tuned for prob's pattern in the first cache that
    has it, else None."""
    key = pattern_key(prob, precision)
    for path in paths:
        e = load_cache(path).get(key) if path else None
        if e is not None:
            return int(e["leaf_nodes"]), int(e["panel"])
    return None


@dataclass(frozen=True)
class Choice:
    leaf_nodes: int
    panel: int
    ms: float


def _pattern(prob):
    """(dim, n_nodes, n_elem, conn, fixed) of a problem or of a list of
    batched instances joined in order (node ids shifted as sgn_batch_setup
    shifts them)."""
    if isinstance(prob, (list, tuple)):
        off, conns = 0, []
        for pr in prob:
            conns.append(np.asarray(pr.conn, dtype=np.int64) + off)
            off += pr.n_nodes
        conn = np.concatenate(conns).astype(np.int32)
        fixed = np.concatenate([np.asarray(pr.fixed_node, dtype=np.uint8) for pr in prob])
        return prob[0].dim, off, conn.shape[0], conn, fixed
    return prob.dim, prob.n_nodes, prob.n_elem, prob.conn, prob.fixed_node


def pattern_key(prob, precision) -> str:
    """Hash of what the symbolic phase sees: dimension, connectivity, fixed
    nodes (and the precision the step runs in)."""
    dim, n_nodes, n_elem, conn, fixed = _pattern(prob)
    h = hashlib.sha256()
    h.update(np.int64([dim, n_nodes, n_elem, int(precision)]).tobytes())
    h.update(np.ascontiguousarray(conn, dtype=np.int32).tobytes())
    h.update(np.ascontiguousarray(fixed, dtype=np.uint8).tobytes())
    return h.hexdigest()[:32]


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(path: str, cache: dict) -> None:
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def candidates(dim: int, panels=PANELS, leaves=LEAVES):
    """Candidate (leaf_nodes, panel) pairs.  A 3D front's fully-summed block
    holds 2 d = 6 unknowns per node, a 2D one 4, so leaves far below one panel
    only add launches; pairs whose leaf front is under half a panel are
    skipped."""
    per_node = 4 * dim // 2  # (x, lambda) pair per coordinate
    out = []
    for leaf in leaves:
        for panel in panels:
            if leaf * per_node * 2 < panel:
                continue
            out.append((leaf, panel))
    return out


def choose(timings):
    """The fastest (leaf, panel) of {(leaf, panel): ms}; ties go to the
    earlier candidate."""
    best = None
    for (leaf, panel), ms in timings.items():
        if best is None or ms < best.ms:
            best = Choice(leaf, panel, ms)
    return best


def measure_step(P, prob, precision, leaf, panel, x=None, reps=5, warmup=2, refine_steps=4):
    """ms per graph-captured SGN step of prob with these set-up options
    (CUDA events on the step's stream, after warm-up launches)."""
    import torch
    stores = B.STORE_MIXED if precision == B.MIXED else B.STORE_FP64
    batched = isinstance(prob, (list, tuple))
    if batched:
        s = P.SGN.from_batch(prob, stores=stores, leaf_nodes=leaf, panel=panel)
        p0 = np.concatenate([pr.p0 for pr in prob])
    else:
        s = P.SGN.from_problem(prob, stores=stores, leaf_nodes=leaf, panel=panel)
        p0 = prob.p0
    try:
        xs = s.X if x is None else x
        xd = torch.as_tensor(np.ascontiguousarray(xs, dtype=np.float64), device=s.device)
        pd = torch.as_tensor(np.ascontiguousarray(p0, dtype=np.float64), device=s.device)
        out = (torch.empty_like(xd), torch.empty_like(pd), torch.empty_like(xd))
        for _ in range(warmup):
            s.step_graph(xd, pd, precision, refine_steps=refine_steps, out=out, residual=False)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for _ in range(reps):
            s.step_graph(xd, pd, precision, refine_steps=refine_steps, out=out, residual=False)
        e1.record(s.stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps
    finally:
        s.close()
        del s
        torch.cuda.empty_cache()


def tune(P, prob, precision=B.MIXED, cache_path: str | None = DEFAULT_CACHE, x=None, cands=None, force=False,
         measure=None, **measure_kw):
    """Best (leaf_nodes, panel) for prob's pattern; cached in cache_path
    (None: no cache).  x: the positions the step is taken at (default: the
    rest shape).  measure(P, prob, precision, leaf, panel, x=..., **kw) -> ms
    defaults to measure_step."""
    key = pattern_key(prob, precision)
    if cache_path and not force:
        e = load_cache(cache_path).get(key)
        if e is not None:
            return Choice(int(e["leaf_nodes"]), int(e["panel"]), float(e["ms"]))
    measure = measure or measure_step
    timings = {}
    dim = prob[0].dim if isinstance(prob, (list, tuple)) else prob.dim
    for leaf, panel in (cands or candidates(dim)):
        timings[(leaf, panel)] = float(measure(P, prob, precision, leaf, panel, x=x, **measure_kw))
    best = choose(timings)
    if cache_path:
        cache = load_cache(cache_path)
        name = f"{len(prob)} instances" if isinstance(prob, (list, tuple)) else prob.name
        cache[key] = {"leaf_nodes": best.leaf_nodes, "panel": best.panel, "ms": best.ms, "name": name,
                      "timings": {f"{l}/{p}": t for (l, p), t in timings.items()}}
        store_cache(cache_path, cache)
    return best


def main(argv=None):
    """python -m paper_2107_03285_gb300.autotune --workload kuhn3d_40 [--precision mixed] [--out PATH]"""
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", action="append", required=True)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--out", default=SHIPPED)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args(argv)
    import paper_2107_03285_gb300 as P
    from sgn_inputs import make_preset
    prec = B.MIXED if args.precision == "mixed" else B.FP64
    for wl in args.workload:
        prob = make_preset(wl)
        best = tune(P, prob, prec, cache_path=args.out, force=True, reps=args.reps)
        print(json.dumps({"workload": wl, "leaf_nodes": best.leaf_nodes, "panel": best.panel, "ms": best.ms}))


if __name__ == "__main__":
    main()
