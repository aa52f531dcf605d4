"""Sharding of independent instances over ranks (paper_2107_03285_gb300/shard.py):
two gloo ranks on CPU partition a batch by estimated cost, build their own
sub-batches and reduce a timing; together they must cover every instance
exactly once, with balanced loads, and agree on the assignment."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2107_03285_gb300 import shard  # noqa: E402
from sgn_inputs import problem_batch2d, select_instances  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = problem_batch2d(24, seed=3, side_lo=5, side_hi=30)
    parts = shard.partition(shard.instance_costs(b.meta["sides"]), world)
    mine = parts[rank]
    sub = select_instances(b, mine)
    got = [None] * world
    dist.all_gather_object(got, ([int(i) for i in mine], sub.n_nodes, sub.n_elem))
    t = shard.max_over_ranks(float(rank + 1))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, t))


def test_partition_is_a_balanced_disjoint_cover():
    costs = shard.instance_costs(np.random.default_rng(0).integers(10, 61, size=256))
    for n in (1, 2, 4, 8):
        parts = shard.partition(costs, n)
        allidx = np.concatenate(parts)
        assert sorted(allidx.tolist()) == list(range(256))
        loads = [costs[p].sum() for p in parts]
        assert max(loads) <= 1.05 * min(loads)
    # deterministic
    assert all((a == b).all() for a, b in zip(shard.partition(costs, 4), shard.partition(costs, 4)))


def test_selected_instances_keep_their_data():
    b = problem_batch2d(12, seed=7, side_lo=5, side_hi=24)
    sel = [3, 0, 7]
    s = select_instances(b, sel)
    no, so = b.meta["node_offsets"], s.meta["node_offsets"]
    eo, seo = b.meta["elem_offsets"], s.meta["elem_offsets"]
    for k, i in enumerate(sel):
        np.testing.assert_array_equal(s.X[so[k]:so[k + 1]], b.X[no[i]:no[i + 1]])
        np.testing.assert_array_equal(s.p0[seo[k]:seo[k + 1]], b.p0[eo[i]:eo[i + 1]])
        np.testing.assert_array_equal(s.conn[seo[k]:seo[k + 1]] - so[k], b.conn[eo[i]:eo[i + 1]] - no[i])
    assert s.track_dof.size == s.target.size == s.weight.size
    assert s.n_nodes == sum(no[i + 1] - no[i] for i in sel)


def test_two_gloo_ranks_cover_the_batch():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {r: (got, t) for r, got, t in (q.get(timeout=120) for _ in procs)}
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got0, t0 = out[0]
    got1, t1 = out[1]
    assert got0 == got1 and t0 == t1 == 2.0
    idx = sorted(got0[0][0] + got0[1][0])
    b = problem_batch2d(24, seed=3, side_lo=5, side_hi=30)
    assert idx == list(range(24))
    assert got0[0][1] + got0[1][1] == b.n_nodes
    assert got0[0][2] + got0[1][2] == b.n_elem
