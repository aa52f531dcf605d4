"""Python front end of the learned warm start (include/sgn_learn.h).

The equilibrium x(p) is recomputed by Newton's method after every design
update (Sec. 5, "Computing Equilibrium States").  ``WarmStart`` predicts the
starting point from the RBF design coefficients theta (p = Phi theta):
x0 = X + u_bar + U c(theta), with u_bar, U from a randomised SVD of
displacement snapshots and c(theta) a BF16 MLP trained with AdamW, all in
libsgn's CUDA kernels.  This module only marshals arguments.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import binding as B


class WarmStart:
    def __init__(self, sgn, centers, width, n_modes=128, hidden=512, max_snap=512, batch=64):
        torch = sgn._torch
        self._torch = torch
        self.sgn = sgn
        self.lib = sgn.lib
        self.centers = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, sgn.dim)
        self.n_rbf = self.centers.shape[0]
        self.n_modes, self.hidden, self.batch = int(n_modes), int(hidden), int(batch)
        opts = B.LearnOpts(self.n_rbf, B._dptr(self.centers, C.c_double), float(width), self.n_modes,
                           self.hidden, int(max_snap), self.batch)
        h = C.c_void_p()
        self._chk(self.lib.sgn_learn_create(sgn.h, C.byref(opts), C.byref(h)), "sgn_learn_create")
        self.h = h
        nbytes = C.c_size_t()
        self._chk(self.lib.sgn_learn_device_bytes(self.h, C.byref(nbytes)), "sgn_learn_device_bytes")
        self.buf = torch.empty(int(nbytes.value), dtype=torch.uint8, device=sgn.device)
        self._chk(self.lib.sgn_learn_bind(self.h, C.c_void_p(self.buf.data_ptr()), int(nbytes.value)),
                  "sgn_learn_bind")
        self.n_params = int(self.lib.sgn_learn_param_count(self.h))

    def _chk(self, code, where):
        return B._check(code, where, self.sgn.h)

    def close(self):
        if getattr(self, "h", None):
            self._torch.cuda.synchronize(self.sgn.device)
            self.lib.sgn_learn_destroy(self.h)
            self.h = None
            self.buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, a, shape):
        return self.sgn._dev(a, shape)

    # ------------------------------------------------------------------ C ABI
    def rbf_params(self, theta):
        th = self._dev(theta, (self.n_rbf,))
        p = self.sgn._empty(self.sgn.n_elem)
        self._chk(self.lib.sgn_rbf_params(self.h, self.sgn._p(th), self.sgn._p(p)), "sgn_rbf_params")
        return p

    def fit_basis(self, snaps, seed=0):
        """snaps: (n_snap, n_nodes, dim) displacements; returns sigma (n_modes,)."""
        S = self._dev(snaps, (-1, self.sgn.n_nodes, self.sgn.dim))
        sigma = np.zeros(self.n_modes)
        self._chk(self.lib.sgn_learn_basis(self.h, self.sgn._p(S), int(S.shape[0]), int(seed),
                                           B._dptr(sigma, C.c_double)), "sgn_learn_basis")
        return sigma

    def train(self, thetas, snaps, steps, lr=1e-3, weight_decay=1e-4, seed=0):
        th = self._dev(thetas, (-1, self.n_rbf))
        S = self._dev(snaps, (-1, self.sgn.n_nodes, self.sgn.dim))
        if th.shape[0] != S.shape[0]:
            raise ValueError("one theta per snapshot")
        loss = C.c_float(0.0)
        self._chk(self.lib.sgn_learn_train(self.h, self.sgn._p(th), self.sgn._p(S), int(S.shape[0]), int(steps),
                                           float(lr), float(weight_decay), int(seed), C.byref(loss)),
                  "sgn_learn_train")
        return loss.value

    def predict(self, theta):
        th = self._dev(theta, (self.n_rbf,))
        x0 = self.sgn._empty(self.sgn.n_nodes, self.sgn.dim)
        self._chk(self.lib.sgn_learn_predict(self.h, self.sgn._p(th), self.sgn._p(x0)), "sgn_learn_predict")
        return x0

    def equilibrium(self, theta, fext, x_prev=None, max_iter=0, tol=0.0, precision=B.FP64):
        """Newton equilibrium at p = Phi theta from the better of the learned
        warm start and x_prev (None: the rest shape).  Returns (x, report,
        used_warm_start)."""
        s = self.sgn
        th = self._dev(theta, (self.n_rbf,))
        fd = self._dev(fext, (s.n_nodes, s.dim))
        xp = self._dev(x_prev, (s.n_nodes, s.dim)) if x_prev is not None else None
        x = s._empty(s.n_nodes, s.dim)
        rep = B.NewtonReport()
        used = C.c_int32(0)
        opts = B.NewtonOpts(int(max_iter), float(tol), int(precision))
        code = self.lib.sgn_equilibrium_warm(self.h, s._p(th), s._p(fd), s._p(xp), s._p(x), C.byref(opts),
                                             C.byref(rep), C.byref(used))
        if code not in (B.OK, B.ENEWTON):
            self._chk(code, "sgn_equilibrium_warm")
        return x, rep, bool(used.value)

    # ------------------------------------------------------- inspection / tests
    def params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        self._chk(self.lib.sgn_learn_params(self.h, B._dptr(out, C.c_float), 0), "sgn_learn_params")
        return out

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32).reshape(-1)
        if a.size != self.n_params:
            raise ValueError("parameter count mismatch")
        self._chk(self.lib.sgn_learn_params(self.h, B._dptr(a, C.c_float), 1), "sgn_learn_params")

    def grads(self, x, t):
        """Loss 1/(2n) sum ||MLP(x) - t||^2 and its parameter gradients."""
        xa = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, self.n_rbf)
        ta = np.ascontiguousarray(t, dtype=np.float32).reshape(-1, self.n_modes)
        g = np.empty(self.n_params, dtype=np.float32)
        loss = C.c_float(0.0)
        self._chk(self.lib.sgn_learn_grads(self.h, B._dptr(xa, C.c_float), B._dptr(ta, C.c_float), xa.shape[0],
                                           C.byref(loss), B._dptr(g, C.c_float)), "sgn_learn_grads")
        return loss.value, g

    def apply(self, grads, lr, weight_decay):
        g = np.ascontiguousarray(grads, dtype=np.float32).reshape(-1)
        self._chk(self.lib.sgn_learn_apply(self.h, B._dptr(g, C.c_float), float(lr), float(weight_decay)),
                  "sgn_learn_apply")

    def basis(self):
        nd = self.sgn.n_nodes * self.sgn.dim
        mean = np.empty(nd)
        U = np.empty((self.n_modes, nd))
        self._chk(self.lib.sgn_learn_basis_get(self.h, B._dptr(mean, C.c_double), B._dptr(U, C.c_double)),
                  "sgn_learn_basis_get")
        return mean, U.T

    def split(self, flat):
        """Flat parameter vector -> [W1, b1, W2, b2, W3, b3] (W as (out, in))."""
        H, nr, nm = self.hidden, self.n_rbf, self.n_modes
        shapes = [(H, nr), (H,), (H, H), (H,), (nm, H), (nm,)]
        out, o = [], 0
        for s in shapes:
            n = int(np.prod(s))
            out.append(np.asarray(flat[o:o + n]).reshape(s))
            o += n
        return out
