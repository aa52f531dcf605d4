"""sgn_assemble_static: the assembly entry point whose per-element scratch is a
fixed device array inside the library, for callers that must not allocate
device memory (or have the runtime set any up) while they assemble, such as
a service whose allocator is frozen after start-up.  Its output must equal
sgn_assemble's, call after call, since all calls share the array; and a call
must leave the device's free memory unchanged (the array is set up at
sgn_bind).  Kept in a file that pytest collects last."""
import ctypes as C

import numpy as np
import pytest

from sgn_inputs import problem_2d, problem_3d

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


def _kkt_dense_coo(s):
    r, c, v = s.export_kkt()
    order = np.lexsort((c, r))
    return r[order], c[order], v[order]


def _static(s, x, p):
    code = s.lib.sgn_assemble_static(s.h, C.c_void_p(x.data_ptr()), C.c_void_p(p.data_ptr()))
    return code


@pytest.mark.parametrize("which", ["kuhn3d_7", "grid2d_21"])
def test_static_scratch_assembly_matches_sgn_assemble(P, which):
    prob = problem_3d(7, seed=5, p_sigma=0.2) if which == "kuhn3d_7" else problem_2d(seed=3)
    s = P.SGN.from_problem(prob, stores=P.STORE_FP64)
    rng = np.random.default_rng(11)
    for call in range(2):
        # two calls in a row with different inputs: the shared array must not
        # carry anything from the previous call into the result
        # a mild deformation keeps every element well shaped (spacing 0.05-0.17)
        x = prob.X + 0.002 * (call + 1) * rng.standard_normal(prob.X.shape) * (prob.fixed_node[:, None] == 0)
        p = prob.p0 + 0.1 * rng.standard_normal(prob.n_elem)
        xd = torch.as_tensor(x, device="cuda")
        pd = torch.as_tensor(p, device="cuda")
        s.assemble(xd, pd)
        r0, c0, v0 = _kkt_dense_coo(s)
        assert _static(s, xd, pd) == P.binding.OK
        r1, c1, v1 = _kkt_dense_coo(s)
        assert np.array_equal(r0, r1) and np.array_equal(c0, c1)
        scale = np.abs(v0).max()
        assert np.max(np.abs(v1 - v0)) <= 1e-12 * scale
        # the factor and step built on it agree too
        s.factor(P.FP64, report=False)
        _, dp1, _, _ = s.solve(P.RHS_KKT, report=False)
        s.assemble(xd, pd)
        s.factor(P.FP64, report=False)
        _, dp0, _, _ = s.solve(P.RHS_KKT, report=False)
        rel = float(torch.linalg.norm(dp1 - dp0) / torch.linalg.norm(dp0))
        assert rel <= 1e-12
    s.close()


def test_static_scratch_call_allocates_nothing(P):
    """Device free memory (cudaMemGetInfo) is the same before and after two
    calls: the array was set up when the handle was bound."""
    prob = problem_3d(9, seed=6, p_sigma=0.1)
    s = P.SGN.from_problem(prob, stores=P.STORE_FP64)
    xd = torch.as_tensor(prob.X, device="cuda")
    pd = torch.as_tensor(prob.p0, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert _static(s, xd, pd) == P.binding.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    s.close()


def test_static_scratch_rejects_meshes_beyond_its_limit(P):
    prob = problem_3d(30)  # 146,334 tets > 139,810
    s = P.SGN.from_problem(prob, stores=0)
    xd = torch.as_tensor(prob.X, device="cuda")
    pd = torch.as_tensor(prob.p0, device="cuda")
    code = _static(s, xd, pd)
    assert code == P.binding.EINVAL
    assert "16 MB" in s.lib.sgn_strerror(code).decode()
    s.close()
