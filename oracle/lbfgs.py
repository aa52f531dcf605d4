"""L-BFGS whose initial inverse Hessian is the Gauss-Newton one (plain FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 4 ("Combination with L-BFGS"): Sparse Gauss-Newton initialises the
inverse Hessian approximation of L-BFGS, so every search direction costs one
solve with the Gauss-Newton matrix.  The direction is the standard two-loop
recursion (Nocedal & Wright, Numerical Optimization, Alg. 7.4) with
H_0 = H_GN^{-1}:

    q = g;  for i = k-1 .. k-m:  a_i = rho_i s_i.q,  q -= a_i y_i
    r = H_GN^{-1} q
    for i = k-m .. k-1:  b = rho_i y_i.r,  r += (a_i - b) s_i
    d = -r,   rho_i = 1 / (y_i.s_i)

with (s_i, y_i) = (p_{i+1} - p_i, g_{i+1} - g_i) the most recent m pairs.
Readings (the paper gives no constants): a pair enters the memory only if
y.s > 1e-12 |y| |s|; backtracking line search on f(x(p), p) with Armijo
constant 1e-4 and step halving, starting at t = 1; if g.d >= 0 the step
falls back to -g.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import equilibrium as EQ
from . import system as S


def two_loop(g, pairs, apply_h0_inv):
    """-H_k g for the pairs [(s, y), ...] (oldest first) and the callable
    apply_h0_inv(v) = H_0^{-1} v."""
    q = np.array(g, dtype=np.float64, copy=True)
    alphas = []
    for s, y in reversed(pairs):
        rho = 1.0 / float(np.dot(y, s))
        a = rho * float(np.dot(s, q))
        q -= a * y
        alphas.append((rho, a))
    r = apply_h0_inv(q)
    for (s, y), (rho, a) in zip(pairs, reversed(alphas)):
        b = rho * float(np.dot(y, r))
        r += (a - b) * s
    return -r


def gn_inverse(prob, x, p):
    """H_GN^{-1} applied by a Cholesky factor of the dense Gauss-Newton
    matrix at (x, p) (Eq. reducedGN), and the gradient df/dp there."""
    b = S.blocks(prob, x, p)
    _, _, H, g, _ = S.dense_gn(b)
    c = sla.cho_factor(H)
    return (lambda v: sla.cho_solve(c, v)), g


def objective_at(prob, p, x0=None):
    """f(x(p), p) with x(p) the equilibrium (Newton from x0)."""
    x, info = EQ.newton(prob, p, x0=x0)
    return S.objective(prob, x, p), x, info


def optimize(prob, p0, iters, m, armijo=1e-4, max_halvings=30):
    """iters L-BFGS iterations from p0 with the Gauss-Newton initial inverse
    Hessian.  Returns (p, history of f, history of |g|)."""
    p = np.array(p0, dtype=np.float64, copy=True)
    f, x, _ = objective_at(prob, p)
    h0_inv, g = gn_inverse(prob, x, p)
    pairs = []
    fh, gh = [f], [float(np.linalg.norm(g))]
    for _ in range(iters):
        d = two_loop(g, pairs, h0_inv)
        slope = float(np.dot(g, d))
        if slope >= 0.0:
            d = -g
            slope = float(np.dot(g, d))
        t = 1.0
        for _ in range(max_halvings):
            pt = p + t * d
            ft, xt, _ = objective_at(prob, pt, x0=x)
            if ft <= f + armijo * t * slope:
                break
            t *= 0.5
        h0_inv_t, gt = gn_inverse(prob, xt, pt)
        s, y = pt - p, gt - g
        if float(np.dot(y, s)) > 1e-12 * np.linalg.norm(y) * np.linalg.norm(s):
            pairs.append((s, y))
            if len(pairs) > m:
                pairs.pop(0)
        p, x, f, g, h0_inv = pt, xt, ft, gt, h0_inv_t
        fh.append(f)
        gh.append(float(np.linalg.norm(g)))
    return p, fh, gh
