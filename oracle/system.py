"""Assembled derivatives, the saddle-point system and dense Gauss-Newton.

Unknowns: x = positions of the free nodes (n_x = d * n_free, free nodes in
their original order, node-major), p = per-element log-moduli (n_p = n_e),
lambda = multipliers, one per equilibrium equation (n_c = n_x).

Objective (Eq. leastSquaresObjective with residuals r = sqrt(w)(x_t - target)
on the tracked coordinates and r = sqrt(alpha) p):
    f(x, p) = 1/2 sum_t w_t (x_t - target_t)^2 + alpha/2 ||p||^2,
so A = sum_i w_i dr_i/dx^T dr_i/dx = diag(w on tracked DOFs),
B = sum_i w_i dr_i/dp^T dr_i/dx = 0 and C = alpha I (Eq. reducedGN).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import elements as el


@dataclass
class Blocks:
    K: sp.csr_matrix        # dc/dx   (n_x, n_x), symmetric
    cp: sp.csr_matrix       # dc/dp   (n_x, n_p)
    A: sp.csr_matrix        # d2f/dx2 (n_x, n_x), diagonal
    C: sp.csr_matrix        # d2f/dp2 (n_p, n_p) = alpha I
    fx: np.ndarray          # df/dx   (n_x,)
    fp: np.ndarray          # df/dp   (n_p,)
    c: np.ndarray           # constraint residual f_int - f_ext (n_x,)


def free_dof_map(prob):
    """Global DOF node*d+comp -> free DOF index (or -1)."""
    d = prob.dim
    free_nodes = np.nonzero(prob.fixed_node == 0)[0]
    node_to_free = -np.ones(prob.n_nodes, dtype=np.int64)
    node_to_free[free_nodes] = np.arange(free_nodes.shape[0])
    g2f = -np.ones(prob.n_nodes * d, dtype=np.int64)
    for k in range(d):
        ok = node_to_free >= 0
        g2f[np.nonzero(ok)[0] * d + k] = node_to_free[ok] * d + k
    return g2f


def positions_from_free(prob, xf):
    """Full node positions: free DOFs from xf, fixed nodes at rest."""
    g2f = free_dof_map(prob)
    x = prob.X.reshape(-1).astype(xf.dtype).copy()
    m = g2f >= 0
    x[m] = xf[g2f[m]]
    return x.reshape(prob.X.shape)


def displacements_from_free(prob, uf):
    """Full node displacements: free DOFs from uf, fixed nodes zero."""
    g2f = free_dof_map(prob)
    u = np.zeros(prob.X.size, dtype=uf.dtype)
    m = g2f >= 0
    u[m] = uf[g2f[m]]
    return u.reshape(prob.X.shape)


def free_from_positions(prob, x):
    g2f = free_dof_map(prob)
    xf = np.empty(int(np.count_nonzero(g2f >= 0)), dtype=x.dtype)
    m = g2f >= 0
    xf[g2f[m]] = x.reshape(-1)[m]
    return xf


def element_dofs(prob):
    """(n_e, (d+1) d) free-DOF index of every element DOF, -1 if fixed."""
    g2f = free_dof_map(prob)
    d = prob.dim
    gl = prob.conn[:, :, None].astype(np.int64) * d + np.arange(d)[None, None, :]
    return g2f[gl.reshape(prob.n_elem, -1)]


def moduli(prob, p):
    return prob.E0 * np.exp(p)


def potential(prob, x, p, u=None):
    """Pi(x; p) = sum_e vol_e Psi(F_e) - f_ext . x (fixed nodes contribute
    a constant).  Given displacements u (x = X + u) instead, the constant
    f_ext . X is left out: Pi = sum_e vol_e Psi(F_e) - f_ext . u."""
    E = moduli(prob, p)
    if u is not None:
        W = el.element_energy(None, prob.X, prob.conn, E, prob.nu, u=u)
        return W.sum() - np.sum(prob.fext * u)
    W = el.element_energy(x, prob.X, prob.conn, E, prob.nu)
    return W.sum() - np.sum(prob.fext * x)


def internal_force(prob, x, p, u=None):
    """Assembled f_int over free DOFs (at positions x, or displacements u)."""
    E = moduli(prob, p)
    fe = el.element_force(x, prob.X, prob.conn, E, prob.nu, u=u).reshape(prob.n_elem, -1)
    dofs = element_dofs(prob)
    n_x = prob.n_free * prob.dim
    out = np.zeros(n_x, dtype=fe.dtype)
    m = dofs >= 0
    np.add.at(out, dofs[m], fe[m])
    return out


def constraint(prob, x, p, u=None):
    """c(x, p) = f_int(x, p) - f_ext on the free DOFs (Eq. optProb)."""
    return internal_force(prob, x, p, u=u) - free_from_positions(prob, prob.fext)


def stiffness(prob, x, p, u=None):
    """K = dc/dx (sparse, free DOFs)."""
    E = moduli(prob, p)
    He = el.element_hessian(x, prob.X, prob.conn, E, prob.nu, u=u)
    nd = (prob.dim + 1) * prob.dim
    He = He.reshape(prob.n_elem, nd, nd)
    dofs = element_dofs(prob)
    rows = np.repeat(dofs[:, :, None], nd, axis=2)
    cols = np.repeat(dofs[:, None, :], nd, axis=1)
    m = (rows >= 0) & (cols >= 0)
    n_x = prob.n_free * prob.dim
    return sp.coo_matrix((He[m], (rows[m], cols[m])), shape=(n_x, n_x)).tocsr()


def param_jacobian(prob, x, p):
    """dc/dp: column e is the force of element e alone (E = E0 e^p and Psi
    linear in E)."""
    E = moduli(prob, p)
    fe = el.element_force(x, prob.X, prob.conn, E, prob.nu).reshape(prob.n_elem, -1)
    dofs = element_dofs(prob)
    cols = np.repeat(np.arange(prob.n_elem)[:, None], dofs.shape[1], axis=1)
    m = dofs >= 0
    n_x = prob.n_free * prob.dim
    return sp.coo_matrix((fe[m], (dofs[m], cols[m])), shape=(n_x, prob.n_elem)).tocsr()


def tracked_free(prob):
    g2f = free_dof_map(prob)
    tf = g2f[prob.track_dof]
    if np.any(tf < 0):
        raise ValueError("tracked DOFs must be free")
    return tf


def objective(prob, x, p):
    xf = x.reshape(-1)
    r = xf[prob.track_dof] - prob.target
    return 0.5 * np.sum(prob.weight * r * r) + 0.5 * prob.alpha * np.dot(p, p)


def blocks(prob, x, p) -> Blocks:
    n_x = prob.n_free * prob.dim
    tf = tracked_free(prob)
    a = np.zeros(n_x)
    np.add.at(a, tf, prob.weight)
    fx = np.zeros(n_x)
    r = x.reshape(-1)[prob.track_dof] - prob.target
    np.add.at(fx, tf, prob.weight * r)
    return Blocks(K=stiffness(prob, x, p), cp=param_jacobian(prob, x, p),
                  A=sp.diags(a).tocsr(), C=(prob.alpha * sp.identity(prob.n_elem)).tocsr(),
                  fx=fx, fp=prob.alpha * p, c=constraint(prob, x, p))


def kkt_matrix(b: Blocks) -> sp.csc_matrix:
    """Eq. sparseSystemGN with the paper's B = d2f/dpdx = 0 here:
        [[A, 0, K^T], [0, C, cp^T], [K, cp, 0]]."""
    return sp.bmat([[b.A, None, b.K.T], [None, b.C, b.cp.T], [b.K, b.cp, None]],
                   format="csc")


def total_gradient(b: Blocks) -> np.ndarray:
    """df/dp = f_p + S^T f_x with S = -K^{-1} cp, computed with one solve
    against K^T (Eq. totalGradient and the remark after it)."""
    lam_adj = adjoint(b)
    return b.fp + b.cp.T @ lam_adj


def adjoint(b: Blocks) -> np.ndarray:
    """lambda = -(dc/dx)^{-T} df/dx^T (Appendix A, Theorem 2)."""
    return -spla.spsolve(b.K.T.tocsc(), b.fx)


def rhs(b: Blocks, mode: str, g=None):
    """'paper': [0; -df/dp; 0] (Eq. sparseSystemGN); 'kkt': [-f_x; -f_p; 0]
    (the Newton-KKT right-hand side of Appendix A)."""
    n_x, n_p = b.K.shape[0], b.C.shape[0]
    if mode == "paper":
        if g is None:
            g = total_gradient(b)
        return np.concatenate([np.zeros(n_x), -g, np.zeros(n_x)])
    if mode == "kkt":
        return np.concatenate([-b.fx, -b.fp, np.zeros(n_x)])
    raise ValueError(mode)


def split(b: Blocks, z):
    n_x, n_p = b.K.shape[0], b.C.shape[0]
    return z[:n_x], z[n_x:n_x + n_p], z[n_x + n_p:]


def sgn_step(b: Blocks, mode="kkt"):
    """Sparse Gauss-Newton step: solve Eq. sparseSystemGN with SuperLU.
    Returns (dx, dp, dlambda)."""
    M = kkt_matrix(b)
    z = spla.splu(M).solve(rhs(b, mode))
    return split(b, z)


def sensitivity(b: Blocks) -> np.ndarray:
    """Dense S = dx/dp = -(dc/dx)^{-1} dc/dp (Eq. dxdp)."""
    Kd = b.K.toarray()
    return -sla.solve(Kd, b.cp.toarray(), assume_a="sym")


def dense_gn(b: Blocks):
    """Dense Gauss-Newton (Eq. reducedGN, Eq. newtonStep):
    H = S^T A S + B S + S^T B^T + C with B = 0, g = df/dp, dp = -H^{-1} g.
    Returns (dp, dx = S dp, H, g, S)."""
    S = sensitivity(b)
    H = S.T @ (b.A @ S) + b.C.toarray()
    g = b.fp + S.T @ b.fx
    c, low = sla.cho_factor(H)
    dp = -sla.cho_solve((c, low), g)
    return dp, S @ dp, H, g, S


def step_error_bound(b: Blocks, dp, g=None, k_solve=None):
    """A-posteriori bound on a computed GN step: with H = S^T A S + alpha I
    and A >= 0 we have H >= alpha I, hence ||dp - dp*|| <= ||H dp + g|| / alpha.
    H dp is applied matrix-free with two solves against K.  Returns
    (bound, ||H dp + g||)."""
    if k_solve is None:
        lu = spla.splu(b.K.tocsc())
        k_solve = lu.solve
    if g is None:
        g = b.fp + b.cp.T @ (-k_solve(b.fx))
    v = -k_solve(b.cp @ dp)          # S dp
    w = b.A @ v
    StAw = -(b.cp.T @ k_solve(w))    # S^T A S dp (K symmetric)
    alpha = b.C.diagonal()[0]
    r = StAw + alpha * dp + g
    return np.linalg.norm(r) / alpha, np.linalg.norm(r)


def inertia(M) -> tuple:
    """(#positive, #negative, #zero) eigenvalues of a small dense symmetric
    matrix, from its spectrum."""
    ev = np.linalg.eigvalsh(M.toarray() if sp.issparse(M) else M)
    tol = 1e-10 * np.max(np.abs(ev))
    return int(np.sum(ev > tol)), int(np.sum(ev < -tol)), int(np.sum(np.abs(ev) <= tol))


def regularized_blocks(b: Blocks, delta: float) -> Blocks:
    """The blocks with delta added to A (x diagonal): the matrix M(delta) an
    inertia-corrected factorization solves (Sec. 5, "Solving the saddle point
    problem": diagonal regularization after an inertia test)."""
    n_x = b.K.shape[0]
    return Blocks(K=b.K, cp=b.cp, A=(b.A + delta * sp.identity(n_x)).tocsr(), C=b.C, fx=b.fx, fp=b.fp, c=b.c)


def inertia_corrected(b: Blocks, delta0: float, growth: float = 10.0, max_tries: int = 30):
    """The first delta of 0, delta0, delta0 growth, ... for which the reduced
    Hessian H(delta) = S^T (A + delta I) S + C is positive definite (the
    saddle-point inertia test), and the Gauss-Newton step there:
    (delta, dp, H(delta))."""
    S = sensitivity(b)
    delta = 0.0
    for _ in range(max_tries):
        H = S.T @ ((b.A + delta * sp.identity(b.K.shape[0])) @ S) + b.C.toarray()
        try:
            c = sla.cho_factor(H)
        except np.linalg.LinAlgError:
            delta = delta0 if delta == 0.0 else delta * growth
            continue
        g = b.fp + S.T @ b.fx
        return delta, -sla.cho_solve(c, g), H
    raise RuntimeError("no regularization made the reduced Hessian positive definite")
