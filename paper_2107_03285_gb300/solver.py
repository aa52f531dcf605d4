"""Python front end of libsgn: one SGN context bound to one CUDA device.

PyTorch provides the device buffer the library carves its matrices, fronts and
workspaces from, and the stream the kernels run on.  All arithmetic of the
SGN step (element evaluation, assembly, factorization, solves, refinement,
Newton equilibrium, adjoint gradient) runs in libsgn's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import binding as B


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class SGN:
    """Sparse Gauss-Newton context for one mesh (Sec. 4, Eq. sparseSystemGN)."""

    def __init__(self, dim, X, conn, fixed_node, E0, nu, stores=B.STORE_FP64 | B.STORE_KFACT,
                 leaf_nodes=0, panel=0, update_ctas=0, device="cuda", stream=None):
        import torch
        self._torch = torch
        self.lib = B.lib()
        self.dim = int(dim)
        self.X = _f64(X).reshape(-1, self.dim)
        self.conn = np.ascontiguousarray(conn, dtype=np.int32)
        self.fixed = np.ascontiguousarray(fixed_node, dtype=np.uint8)
        self.n_nodes, self.n_elem = self.X.shape[0], self.conn.shape[0]
        mesh = B.Mesh(self.dim, self.n_nodes, self.n_elem, B._dptr(self.X, C.c_double),
                      B._dptr(self.conn, C.c_int32), B._dptr(self.fixed, C.c_uint8), float(E0), float(nu))
        opts = B.SetupOpts(int(leaf_nodes), int(panel), int(update_ctas))
        h = C.c_void_p()
        B._check(self.lib.sgn_setup(C.byref(mesh), C.byref(opts), C.byref(h)), "sgn_setup")
        self.h = h
        self._bind(stores, device, stream)

    @classmethod
    def from_batch(cls, probs, stores=B.STORE_FP64 | B.STORE_KFACT, leaf_nodes=0, panel=0, update_ctas=0,
                   device="cuda", stream=None):
        """One handle for many independent instances (sgn_batch_setup): the
        meshes and objectives of `probs` joined in order; x, p, fext and the
        step's outputs are the instances' arrays concatenated."""
        self = cls.__new__(cls)
        import torch
        self._torch = torch
        self.lib = B.lib()
        probs = list(probs)
        self.dim = int(probs[0].dim)
        keep = []
        meshes = (B.Mesh * len(probs))()
        objs = (B.Objective * len(probs))()
        for i, pr in enumerate(probs):
            X = _f64(pr.X).reshape(-1, self.dim)
            conn = np.ascontiguousarray(pr.conn, dtype=np.int32)
            fixed = np.ascontiguousarray(pr.fixed_node, dtype=np.uint8)
            tr = np.ascontiguousarray(pr.track_dof, dtype=np.int64)
            tg, wt = _f64(pr.target), _f64(pr.weight)
            keep += [X, conn, fixed, tr, tg, wt]
            meshes[i] = B.Mesh(self.dim, X.shape[0], conn.shape[0], B._dptr(X, C.c_double),
                               B._dptr(conn, C.c_int32), B._dptr(fixed, C.c_uint8), float(pr.E0), float(pr.nu))
            objs[i] = B.Objective(tr.shape[0], B._dptr(tr, C.c_int64), B._dptr(tg, C.c_double),
                                  B._dptr(wt, C.c_double), float(pr.alpha))
        opts = B.SetupOpts(int(leaf_nodes), int(panel), int(update_ctas))
        h = C.c_void_p()
        B._check(self.lib.sgn_batch_setup(len(probs), meshes, objs, C.byref(opts), C.byref(h)), "sgn_batch_setup")
        self.h = h
        self.X = np.concatenate([_f64(pr.X).reshape(-1, self.dim) for pr in probs])
        self.n_nodes, self.n_elem = self.X.shape[0], sum(int(pr.n_elem) for pr in probs)
        self._bind(stores, device, stream)
        return self

    def _bind(self, stores, device, stream):
        import torch
        self.info = B.Info()
        B._check(self.lib.sgn_get_info(self.h, C.byref(self.info)), "sgn_get_info", self.h)
        self.stores = int(stores)
        nbytes = C.c_size_t()
        B._check(self.lib.sgn_device_bytes(self.h, self.stores, C.byref(nbytes)), "sgn_device_bytes", self.h)
        self.device = torch.device(device)
        self.buf = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        B._check(self.lib.sgn_bind(self.h, C.c_void_p(self.buf.data_ptr()), int(nbytes.value), self.stores,
                                   C.c_void_p(self.stream.cuda_stream)), "sgn_bind", self.h)

    def batch_offsets(self):
        """(node offsets, element offsets), n + 1 each, of a batched handle."""
        n = C.c_int32()
        B._check(self.lib.sgn_batch_info(self.h, C.byref(n), None, None), "sgn_batch_info", self.h)
        no = np.empty(n.value + 1, dtype=np.int64)
        eo = np.empty(n.value + 1, dtype=np.int64)
        B._check(self.lib.sgn_batch_info(self.h, C.byref(n), B._dptr(no, C.c_int64), B._dptr(eo, C.c_int64)),
                 "sgn_batch_info", self.h)
        return no, eo

    def batch_residuals(self, kind=B.BATCH_EQUILIBRIUM):
        """Per-instance relative residuals of the last equilibrium (kind 0)
        or saddle-point solve (kind 1)."""
        no, _ = self.batch_offsets()
        out = np.empty(no.shape[0] - 1)
        B._check(self.lib.sgn_batch_residuals(self.h, int(kind), B._dptr(out, C.c_double)), "sgn_batch_residuals",
                 self.h)
        return out

    @classmethod
    def from_problem(cls, prob, **kw):
        s = cls(prob.dim, prob.X, prob.conn, prob.fixed_node, prob.E0, prob.nu, **kw)
        s.set_objective(prob.track_dof, prob.target, prob.weight, prob.alpha)
        return s

    def close(self):
        if getattr(self, "h", None):
            self._torch.cuda.synchronize(self.device)
            self.lib.sgn_destroy(self.h)
            self.h = None
            self.buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ helpers
    def _dev(self, a, shape):
        t = self._torch
        if isinstance(a, t.Tensor):
            if a.device.type != "cuda" or a.dtype != t.float64 or not a.is_contiguous():
                raise ValueError("device arrays must be contiguous float64 CUDA tensors")
            return a
        return t.as_tensor(_f64(a).reshape(shape), device=self.device)

    def _empty(self, *shape):
        return self._torch.empty(*shape, dtype=self._torch.float64, device=self.device)

    @staticmethod
    def _p(t):
        return C.c_void_p(t.data_ptr()) if t is not None else None

    # ---------------------------------------------------------------- C ABI
    def set_objective(self, track_dof, target, weight, alpha):
        self._track = np.ascontiguousarray(track_dof, dtype=np.int64)
        self._target = _f64(target)
        self._weight = _f64(weight)
        obj = B.Objective(self._track.shape[0], B._dptr(self._track, C.c_int64),
                          B._dptr(self._target, C.c_double), B._dptr(self._weight, C.c_double), float(alpha))
        B._check(self.lib.sgn_set_objective(self.h, C.byref(obj)), "sgn_set_objective", self.h)

    def assemble(self, x, p):
        self._x = self._dev(x, (self.n_nodes, self.dim))
        self._pv = self._dev(p, (self.n_elem,))
        B._check(self.lib.sgn_assemble(self.h, self._p(self._x), self._p(self._pv)), "sgn_assemble", self.h)

    def factor(self, precision=B.FP64, report=True, eps_x=0.0, eps_lambda=0.0):
        """LDL^T of the assembled matrix, or (eps_x, eps_lambda > 0) of its
        stabilized form (sgn_factor_ex), which the solves use as a
        preconditioner."""
        rep = B.FactorReport() if report else None
        opts = B.FactorOpts(float(eps_x), float(eps_lambda))
        B._check(self.lib.sgn_factor_ex(self.h, int(precision), C.byref(opts), C.byref(rep) if report else None),
                 "sgn_factor_ex", self.h)
        return rep

    def solve(self, mode=B.RHS_KKT, g=None, max_refine=0, tol=0.0, report=True, out=None, method=B.SOLVE_AUTO,
              max_krylov=0, regularized=False):
        dx, dp, dl = out if out is not None else (self._empty(self.n_nodes, self.dim), self._empty(self.n_elem),
                                                   self._empty(self.n_nodes, self.dim))
        gd = self._dev(g, (self.n_elem,)) if g is not None else None
        opts = B.SolveOpts(int(max_refine), float(tol), int(method), int(max_krylov), int(bool(regularized)))
        rep = B.SolveReport() if report else None
        B._check(self.lib.sgn_solve(self.h, int(mode), self._p(gd), self._p(dx), self._p(dp), self._p(dl),
                                    C.byref(opts), C.byref(rep) if report else None), "sgn_solve", self.h)
        return dx, dp, dl, rep

    def step(self, x, p, precision=B.FP64, mode=B.RHS_KKT, g=None):
        self.assemble(x, p)
        frep = self.factor(precision)
        dx, dp, dl, srep = self.solve(mode, g)
        return dx, dp, dl, frep, srep

    def step_graph(self, x, p, precision=B.MIXED, refine_steps=3, out=None, residual=True):
        """One SGN step as a single CUDA-graph launch (captured on first use
        for these buffers).  x, p must stay the same device tensors between
        calls for the graph to be replayed."""
        x = self._dev(x, (self.n_nodes, self.dim))
        p = self._dev(p, (self.n_elem,))
        dx, dp, dl = out if out is not None else (self._empty(self.n_nodes, self.dim), self._empty(self.n_elem),
                                                   self._empty(self.n_nodes, self.dim))
        res = C.c_double(0.0)
        B._check(self.lib.sgn_step_graph(self.h, int(precision), int(refine_steps), self._p(x), self._p(p),
                                         self._p(dx), self._p(dp), self._p(dl),
                                         C.byref(res) if residual else None), "sgn_step_graph", self.h)
        self._x, self._pv = x, p
        return dx, dp, dl, res.value

    def step_host(self, x, p, precision=B.FP64):
        """Host buffers in and out (H2D / D2H copies inside the call)."""
        xh = _f64(x).reshape(self.n_nodes, self.dim)
        ph = _f64(p).reshape(self.n_elem)
        dx = np.empty_like(xh)
        dl = np.empty_like(xh)
        dp = np.empty_like(ph)
        rep = B.SolveReport()
        dptr = lambda a: B._dptr(a, C.c_double)
        code = self.lib.sgn_step_host(self.h, int(precision), dptr(xh), dptr(ph), dptr(dx), dptr(dp), dptr(dl),
                                      C.byref(rep))
        if code not in (B.OK, B.EREFINE):
            B._check(code, "sgn_step_host", self.h)
        return dx, dp, dl, rep

    def equilibrium(self, p, fext, x0=None, max_iter=0, tol=0.0, precision=B.FP64):
        """Newton equilibrium (K fronts in FP64, or FP32 with FP64-refined
        directions for precision=MIXED, which needs STORE_KFACT_MIXED)."""
        pd = self._dev(p, (self.n_elem,))
        fd = self._dev(fext, (self.n_nodes, self.dim))
        x = self._dev(self.X if x0 is None else x0, (self.n_nodes, self.dim)).clone()
        rep = B.NewtonReport()
        code = self.lib.sgn_equilibrium(self.h, self._p(pd), self._p(fd), self._p(x),
                                        C.byref(B.NewtonOpts(int(max_iter), float(tol), int(precision))),
                                        C.byref(rep))
        if code not in (B.OK, B.ENEWTON):  # non-convergence is reported in rep.converged
            B._check(code, "sgn_equilibrium", self.h)
        return x, rep

    def export_kkt(self):
        """Assembled saddle-point matrix as (rows, cols, vals) host COO arrays."""
        n = C.c_int64()
        B._check(self.lib.sgn_export_kkt(self.h, C.byref(n), None, None, None), "sgn_export_kkt", self.h)
        rows = np.empty(n.value, dtype=np.int64)
        cols = np.empty(n.value, dtype=np.int64)
        vals = np.empty(n.value, dtype=np.float64)
        B._check(self.lib.sgn_export_kkt(self.h, C.byref(n), B._dptr(rows, C.c_int64), B._dptr(cols, C.c_int64),
                                         B._dptr(vals, C.c_double)), "sgn_export_kkt", self.h)
        return rows, cols, vals

    def profile(self, mask=1):
        """Enable CUDA-event timing of the kernel kinds in `mask` (bit k =
        binding.PROF_KINDS[k]); 0 disables.  Resets the timers."""
        B._check(self.lib.sgn_profile(self.h, int(mask)), "sgn_profile", self.h)

    def profile_read(self):
        """{kind: (launches, seconds, flops)} since the last profile()."""
        n = len(B.PROF_KINDS)
        arr = (B.KernelProfile * n)()
        B._check(self.lib.sgn_profile_read(self.h, arr, n), "sgn_profile_read", self.h)
        return {B.PROF_KINDS[k]: (arr[k].launches, arr[k].seconds, arr[k].flops) for k in range(n)}

    def launch_count(self):
        return int(self.lib.sgn_launch_count(self.h))

    def factor_inertia(self, precision=B.FP64, delta0=0.0, growth=0.0, max_tries=0):
        """Inertia-corrected factorization (sgn_factor_inertia): returns
        (delta, factor report)."""
        rep = B.FactorReport()
        delta = C.c_double()
        B._check(self.lib.sgn_factor_inertia(self.h, int(precision), C.byref(B.InertiaOpts(float(delta0),
                                                                                           float(growth),
                                                                                           int(max_tries))),
                                             C.byref(delta), C.byref(rep)), "sgn_factor_inertia", self.h)
        return delta.value, rep

    def objective(self, x, p):
        """f(x, p) of the handle's objective (sgn_objective_value)."""
        f = C.c_double()
        xd = self._dev(x, (self.n_nodes, self.dim))  # kept alive across the call
        pd = self._dev(p, (self.n_elem,))
        B._check(self.lib.sgn_objective_value(self.h, self._p(xd), self._p(pd), C.byref(f)), "sgn_objective_value",
                 self.h)
        return f.value

    def lbfgs_direction(self, S, Y, g):
        """-H_k g over the pairs S, Y ([m][n_elem], oldest first) with the SGN
        inverse of the current factor as H_0 (sgn_lbfgs_direction)."""
        m = 0 if S is None else int(S.shape[0])
        gd = self._dev(g, (self.n_elem,))
        d = self._empty(self.n_elem)
        Sd = self._dev(S, (m, self.n_elem)) if m else None
        Yd = self._dev(Y, (m, self.n_elem)) if m else None
        B._check(self.lib.sgn_lbfgs_direction(self.h, m, self._p(Sd), self._p(Yd), self._p(gd), self._p(d)),
                 "sgn_lbfgs_direction", self.h)
        return d

    def optimize_lbfgs(self, p0, fext, x0=None, m=5, max_iter=10, tol_g=0.0, precision=B.MIXED,
                       eq_precision=B.MIXED):
        """SGN-initialised L-BFGS (sgn_optimize_lbfgs): returns (p, x, report)."""
        p = self._dev(p0, (self.n_elem,)).clone()
        x = self._dev(self.X if x0 is None else x0, (self.n_nodes, self.dim)).clone()
        fd = self._dev(fext, (self.n_nodes, self.dim))
        nbytes = C.c_size_t()
        B._check(self.lib.sgn_lbfgs_work_bytes(self.h, int(m), C.byref(nbytes)), "sgn_lbfgs_work_bytes", self.h)
        work = self._torch.empty(int(nbytes.value), dtype=self._torch.uint8, device=self.device)
        rep = B.LbfgsReport()
        opts = B.LbfgsOpts(int(m), int(max_iter), float(tol_g), int(precision), int(eq_precision), 0.0, 0)
        B._check(self.lib.sgn_optimize_lbfgs(self.h, self._p(fd), self._p(p), self._p(x),
                                             C.c_void_p(work.data_ptr()), int(nbytes.value), C.byref(opts),
                                             C.byref(rep)), "sgn_optimize_lbfgs", self.h)
        return p, x, rep

    def factor_k(self):
        B._check(self.lib.sgn_factor_k(self.h), "sgn_factor_k", self.h)

    def gradient(self):
        g = self._empty(self.n_elem)
        B._check(self.lib.sgn_gradient(self.h, self._p(g)), "sgn_gradient", self.h)
        return g
