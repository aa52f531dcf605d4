"""CPU-side checks of the C ABI: the library builds and loads, exports every
symbol include/sgn.h declares, and its host-only calls (symbolic set-up,
info, device sizing, argument validation) behave.  No GPU needed."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from sgn_inputs import problem_2d, problem_3d, problem_tiny_3d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2107_03285_gb300 import build as build_mod
    build_mod.build()
    from paper_2107_03285_gb300 import binding
    return binding


def _declared_symbols():
    out = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", name)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            out |= set(re.findall(r"\b(sgn_[a-z0-9_]+)\s*\(", txt))
    return out


def test_library_exports_every_declared_symbol(B):
    lib = B.load_library()
    declared = _declared_symbols()
    assert declared, "no declarations found"
    for sym in sorted(declared):
        assert hasattr(lib, sym), sym
    assert declared == set(B.EXPORTED)


def _setup(B, prob, leaf=0, panel=0):
    lib = B.load_library()
    X = np.ascontiguousarray(prob.X, dtype=np.float64)
    conn = np.ascontiguousarray(prob.conn, dtype=np.int32)
    fixed = np.ascontiguousarray(prob.fixed_node, dtype=np.uint8)
    mesh = B.Mesh(prob.dim, X.shape[0], conn.shape[0], B._dptr(X, C.c_double), B._dptr(conn, C.c_int32),
                  B._dptr(fixed, C.c_uint8), prob.E0, prob.nu)
    h = C.c_void_p()
    code = lib.sgn_setup(C.byref(mesh), C.byref(B.SetupOpts(leaf, panel)), C.byref(h))
    return lib, code, h, (X, conn, fixed)


@pytest.mark.parametrize("which", ["grid2d_21", "kuhn3d_5"])
def test_setup_sizes_match_the_oracle_pattern(B, which):
    from oracle import equilibrium as EQ
    from oracle import system as S
    prob = problem_2d() if which == "grid2d_21" else problem_3d(5, p_sigma=0.1)
    lib, code, h, keep = _setup(B, prob)
    assert code == B.OK
    info = B.Info()
    assert lib.sgn_get_info(h, C.byref(info)) == B.OK
    n_x = prob.n_free * prob.dim
    assert info.n_x == n_x and info.n_p == prob.n_elem and info.n_kkt == 2 * n_x + prob.n_elem
    x, _ = EQ.newton(prob, prob.p0)
    M = S.kkt_matrix(S.blocks(prob, x, prob.p0))
    assert info.nnz_kkt + len(np.unique(prob.track_dof)) == M.nnz
    assert info.factor_flops > 0 and info.nnz_factor > 0 and info.n_levels >= 1
    nbytes = C.c_size_t()
    assert lib.sgn_device_bytes(h, B.STORE_FP64 | B.STORE_MIXED | B.STORE_KFACT, C.byref(nbytes)) == B.OK
    assert nbytes.value > 8 * info.nnz_factor
    lib.sgn_destroy(h)


def test_setup_rejects_bad_meshes(B):
    prob = problem_tiny_3d()
    bad = problem_tiny_3d()
    bad.conn = bad.conn.copy()
    bad.conn[0, 0] = bad.n_nodes + 5
    _, code, _, _ = _setup(B, bad)
    assert code == B.EINVAL
    bad2 = problem_tiny_3d()
    bad2.conn = bad2.conn.copy()
    bad2.conn[0, 1] = bad2.conn[0, 0]   # degenerate element
    _, code, _, _ = _setup(B, bad2)
    assert code == B.EINVAL
    allfixed = problem_tiny_3d()
    allfixed.fixed_node = np.ones_like(allfixed.fixed_node)
    _, code, _, _ = _setup(B, allfixed)
    assert code == B.EINVAL
    _, code, _, _ = _setup(B, prob, panel=7)
    assert code == B.EINVAL
    lib = B.load_library()
    assert lib.sgn_setup(None, None, None) == B.EINVAL
    assert lib.sgn_strerror(B.EINVERTED).decode().startswith("inverted")


def test_calls_before_bind_are_rejected(B):
    prob = problem_tiny_3d()
    lib, code, h, keep = _setup(B, prob)
    assert code == B.OK
    assert lib.sgn_assemble(h, None, None) == B.EINVAL
    one = C.c_void_p(1)
    assert lib.sgn_assemble(h, one, one) == B.ESTATE
    assert lib.sgn_factor(h, B.FP64, None) == B.ESTATE
    lib.sgn_destroy(h)


@pytest.mark.parametrize("which", ["kuhn3d_9", "batch2d_12", "kuhn3d_16"])
def test_contribution_block_arena_plan_is_consistent(B, which):
    """sgn_device_bytes replays the contribution-block lifetimes and fails if
    two live blocks would share memory, and checks that every substitution
    schedule lists each front's items after the items they wait on (on the
    16^3 cube also the parts of split backward ancestor-row products: fronts
    below the root have 1,536 ancestor rows); the arena must also need less
    than keeping every front whole."""
    from sgn_inputs import make_preset
    prob = make_preset(which)
    lib, code, h, keep = _setup(B, prob)
    assert code == B.OK
    sizes = {}
    for m in (B.STORE_FP64, B.STORE_MIXED, B.STORE_KFACT, B.STORE_KFACT_MIXED, 15):
        n = C.c_size_t()
        assert lib.sgn_device_bytes(h, m, C.byref(n)) == B.OK
        sizes[m] = n.value
    assert sizes[15] < sizes[B.STORE_FP64] + sizes[B.STORE_MIXED] + sizes[B.STORE_KFACT] + sizes[B.STORE_KFACT_MIXED]
    lib.sgn_destroy(h)


def _batch_setup(B, probs, alphas=None):
    lib = B.load_library()
    keep = []
    meshes = (B.Mesh * len(probs))()
    objs = (B.Objective * len(probs))()
    for i, pr in enumerate(probs):
        X = np.ascontiguousarray(pr.X, dtype=np.float64)
        conn = np.ascontiguousarray(pr.conn, dtype=np.int32)
        fixed = np.ascontiguousarray(pr.fixed_node, dtype=np.uint8)
        tr = np.ascontiguousarray(pr.track_dof, dtype=np.int64)
        tg = np.ascontiguousarray(pr.target, dtype=np.float64)
        wt = np.ascontiguousarray(pr.weight, dtype=np.float64)
        keep += [X, conn, fixed, tr, tg, wt]
        meshes[i] = B.Mesh(pr.dim, X.shape[0], conn.shape[0], B._dptr(X, C.c_double), B._dptr(conn, C.c_int32),
                           B._dptr(fixed, C.c_uint8), pr.E0, pr.nu)
        a = pr.alpha if alphas is None else alphas[i]
        objs[i] = B.Objective(tr.shape[0], B._dptr(tr, C.c_int64), B._dptr(tg, C.c_double),
                              B._dptr(wt, C.c_double), a)
    h = C.c_void_p()
    code = lib.sgn_batch_setup(len(probs), meshes, objs, C.byref(B.SetupOpts(0, 0, 0)), C.byref(h))
    return lib, code, h, keep


def test_batch_setup_joins_instances(B):
    """sgn_batch_setup: offsets of the joined arrays, sizes equal to the sum
    of the instances' own set-ups, overlapping coordinates allowed."""
    from sgn_inputs import batch2d_instances
    probs = batch2d_instances(5, seed=3, side_lo=4, side_hi=9)
    lib, code, h, keep = _batch_setup(B, probs)
    assert code == B.OK
    n = C.c_int32()
    no = np.zeros(6, dtype=np.int64)
    eo = np.zeros(6, dtype=np.int64)
    assert lib.sgn_batch_info(h, C.byref(n), B._dptr(no, C.c_int64), B._dptr(eo, C.c_int64)) == B.OK
    assert n.value == 5
    np.testing.assert_array_equal(no, np.cumsum([0] + [p.n_nodes for p in probs]))
    np.testing.assert_array_equal(eo, np.cumsum([0] + [p.n_elem for p in probs]))
    info = B.Info()
    assert lib.sgn_get_info(h, C.byref(info)) == B.OK
    tot = {"n_x": 0, "nnz_kkt": 0, "nnz_factor": 0}
    for pr in probs:
        l1, c1, h1, k1 = _setup(B, pr)
        assert c1 == B.OK
        i1 = B.Info()
        l1.sgn_get_info(h1, C.byref(i1))
        for k in tot:
            tot[k] += getattr(i1, k)
        l1.sgn_destroy(h1)
    assert info.n_x == tot["n_x"] and info.nnz_kkt == tot["nnz_kkt"]
    # one elimination forest: the factor of the block-diagonal matrix is the
    # union of the instances' factors when every instance keeps its own ordering
    assert info.nnz_factor == tot["nnz_factor"]
    # residuals before any solve: out of order
    out = np.zeros(5)
    assert lib.sgn_batch_residuals(h, 0, B._dptr(out, C.c_double)) == B.ESTATE
    lib.sgn_destroy(h)
    # a plain handle is not a batch
    l2, c2, h2, k2 = _setup(B, probs[0])
    assert l2.sgn_batch_info(h2, C.byref(n), None, None) == B.OK and n.value == 0
    l2.sgn_destroy(h2)


def test_batch_setup_rejects_mismatched_instances(B):
    from sgn_inputs import batch2d_instances, problem_tiny_3d
    probs = batch2d_instances(3, seed=4, side_lo=4, side_hi=6)
    lib, code, h, _ = _batch_setup(B, probs, alphas=[1e-4, 2e-4, 1e-4])
    assert code == B.EINVAL and "alpha" in lib.sgn_strerror(code).decode()
    probs2 = probs[:2] + [problem_tiny_3d()]
    lib, code, h, _ = _batch_setup(B, probs2)
    assert code == B.EINVAL and "dim" in lib.sgn_strerror(code).decode()
    probs[1].E0 = 2e4
    lib, code, h, _ = _batch_setup(B, probs)
    assert code == B.EINVAL
    assert lib.sgn_batch_setup(0, None, None, None, C.byref(C.c_void_p())) == B.EINVAL
