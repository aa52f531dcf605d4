"""Forward simulation: static equilibrium c(x, p) = 0 for fixed p.

Sec. 5 ("Computing Equilibrium States") minimises the simulation's potential
with Newton's method and a backtracking line search that keeps the objective
monotone.  Readings (the paper gives no constants): Armijo constant 1e-4,
step halving, any element with det F <= 0 rejects a trial step, stop when
||c|| <= tol * ||f_ext|| (tol = 1e-10), at most 50 Newton iterations.

The iterate is the displacement u = x - X of the free nodes, and F is formed
from it (F = I + D_u D_m^{-1}): an absolute position carries a
representation error of about eps |x|, which alone puts a floor of a few
1e-10 ||f_ext|| under ||c|| on the meshes here, while a displacement carries
eps |u|.  Measured floors of ||c|| / ||f_ext|| with the displacement
iterate: 1.3e-11 on a 60 x 60 grid (wherever it sits; from absolute
positions 5.2e-10 at the origin and 2.2e-8 at (24, 24)), 8.5e-12 on
40 x 40, 7.6e-14 on a 16^3-node cube.  A caller asking for a tolerance
below the floor would never converge, so a residual that a Newton step no
longer halves also counts as converged once it is below STAGNATION_CAP
||f_ext|| = 1e-10 ||f_ext|| (under 10x the largest floor).  Once the predicted
decrease |t c.dx| is below the round-off of Pi itself (1e-13 |Pi|), a
potential comparison says nothing, and a trial step is accepted when it
lowers ||c|| instead.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import system as S
from . import elements as el

STAGNATION_CAP = 1e-10


def newton(prob, p, x0=None, tol=1e-10, max_iter=50, armijo=1e-4, max_halvings=40):
    """Returns (x, info) with x the full node positions (n_nodes, d) and
    info["u"] the free-DOF displacements the iteration converged to."""
    x_start = prob.X if x0 is None else np.asarray(x0, dtype=np.float64)
    uf = S.free_from_positions(prob, x_start - prob.X)
    fnorm = np.linalg.norm(S.free_from_positions(prob, prob.fext))
    scale = max(fnorm, 1e-300)
    hist = []
    u = S.displacements_from_free(prob, uf)
    Pi = S.potential(prob, None, p, u=u)
    cn_prev = None

    def done(it, converged):
        x = prob.X + S.displacements_from_free(prob, uf)
        c = S.constraint(prob, None, p, u=S.displacements_from_free(prob, uf))
        return x, {"iters": it, "residual": np.linalg.norm(c) / scale, "history": hist,
                   "converged": converged, "u": uf.copy()}

    for it in range(max_iter + 1):
        u = S.displacements_from_free(prob, uf)
        c = S.constraint(prob, None, p, u=u)
        cn = np.linalg.norm(c)
        hist.append(cn / scale)
        stagnated = cn_prev is not None and cn > 0.5 * cn_prev and cn <= STAGNATION_CAP * scale
        if cn <= tol * scale or stagnated:
            return done(it, True)
        cn_prev = cn
        if it == max_iter:
            break
        K = S.stiffness(prob, None, p, u=u)
        du = -spla.spsolve(K.tocsc(), c)
        slope = float(np.dot(c, du))
        t = 1.0
        accepted = False
        for _ in range(max_halvings):
            ut = S.displacements_from_free(prob, uf + t * du)
            J = el.element_jacobian_det(None, prob.X, prob.conn, u=ut)
            if np.all(J > 0):
                Pit = S.potential(prob, None, p, u=ut)
                if Pit <= Pi + armijo * t * slope:
                    accepted = True
                    break
                if abs(t * slope) <= 1e-13 * max(abs(Pi), 1e-300):
                    if np.linalg.norm(S.constraint(prob, None, p, u=ut)) < cn:
                        accepted = True
                        break
            t *= 0.5
        if not accepted:
            # at round-off level the potential can no longer decrease; take the
            # full Newton step if it keeps every element valid
            t = 1.0
            ut = S.displacements_from_free(prob, uf + du)
            if not np.all(el.element_jacobian_det(None, prob.X, prob.conn, u=ut) > 0):
                break
            Pit = S.potential(prob, None, p, u=ut)
        uf, Pi = uf + t * du, Pit
    return done(max_iter, False)
