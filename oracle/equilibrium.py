"""Forward simulation: static equilibrium c(x, p) = 0 for fixed p.

Sec. 5 ("Computing Equilibrium States") minimises the simulation's potential
with Newton's method and a backtracking line search that keeps the objective
monotone.  Readings (the paper gives no constants): Armijo constant 1e-4,
step halving, any element with det F <= 0 rejects a trial step, stop when
||c|| <= tol * ||f_ext|| (tol = 1e-10), at most 50 Newton iterations.  The
round-off floor of ||c|| / ||f_ext|| grows with the mesh (about 5e-10 on a
60 x 60 grid), so a residual that a Newton step no longer halves counts as
converged once it is below 1e-7 ||f_ext|| (stagnation at the floor).  Once
the predicted decrease |t c.dx| is below the round-off of Pi itself
(1e-13 |Pi|), a potential comparison says nothing, and a trial step is
accepted when it lowers ||c|| instead.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import system as S
from . import elements as el


def newton(prob, p, x0=None, tol=1e-10, max_iter=50, armijo=1e-4, max_halvings=40):
    """Returns (x, info) with x the full node positions (n_nodes, d)."""
    x = prob.X.copy() if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    fnorm = np.linalg.norm(S.free_from_positions(prob, prob.fext))
    scale = max(fnorm, 1e-300)
    hist = []
    Pi = S.potential(prob, x, p)
    cn_prev = None
    for it in range(max_iter + 1):
        c = S.constraint(prob, x, p)
        cn = np.linalg.norm(c)
        hist.append(cn / scale)
        stagnated = cn_prev is not None and cn > 0.5 * cn_prev and cn <= 1e-7 * scale
        if cn <= tol * scale or stagnated:
            return x, {"iters": it, "residual": cn / scale, "history": hist, "converged": True}
        cn_prev = cn
        if it == max_iter:
            break
        K = S.stiffness(prob, x, p)
        dx = -spla.spsolve(K.tocsc(), c)
        slope = float(np.dot(c, dx))
        t = 1.0
        xf = S.free_from_positions(prob, x)
        accepted = False
        for _ in range(max_halvings):
            xt = S.positions_from_free(prob, xf + t * dx)
            J = el.element_jacobian_det(xt, prob.X, prob.conn)
            if np.all(J > 0):
                Pit = S.potential(prob, xt, p)
                if Pit <= Pi + armijo * t * slope:
                    accepted = True
                    break
                if abs(t * slope) <= 1e-13 * max(abs(Pi), 1e-300):
                    if np.linalg.norm(S.constraint(prob, xt, p)) < cn:
                        accepted = True
                        break
            t *= 0.5
        if not accepted:
            # at round-off level the potential can no longer decrease; take the
            # full Newton step if it keeps every element valid
            xt = S.positions_from_free(prob, xf + dx)
            if not np.all(el.element_jacobian_det(xt, prob.X, prob.conn) > 0):
                break
            Pit = S.potential(prob, xt, p)
        x, Pi = xt, Pit
    c = S.constraint(prob, x, p)
    return x, {"iters": max_iter, "residual": np.linalg.norm(c) / scale, "history": hist,
               "converged": False}
