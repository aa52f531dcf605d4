"""Compressible neo-Hookean linear simplex elements, FP64 (or complex128 for
complex-step pins), vectorised over elements with plain NumPy.

The paper names linear tetrahedra with a neo-Hookean material for its inverse
elastic design example (Sec. 5, "Inverse Elastic Design") without fixing the
variant.  Reading used throughout (both paths):

    Psi(F) = mu/2 (tr F^T F - d) - mu ln J + lambda/2 (ln J)^2,   J = det F,
    mu = E / (2 (1 + nu)),  lambda = E nu / ((1 + nu)(1 - 2 nu)),
    E_e = E0 exp(p_e)  (p = per-element log Young's modulus).

In 2D the same formula with 2x2 F is plane strain with unit thickness.

Element kinematics: D_m = [X_1 - X_0, ..., X_d - X_0] (columns), vol =
|det D_m| / d!, D_s likewise from the deformed positions, F = D_s D_m^{-1}.
With displacements u = x - X the same F reads F = I + D_u D_m^{-1}
(D_s = D_m + D_u); every element function accepts either positions x or,
through the keyword u, displacements.  The displacement form keeps the
round-off of F independent of where the body sits: an absolute position
carries a representation error of about eps |x|, a displacement one of
eps |u| (the forward simulation iterates on u for that reason).
Writing F_ij = sum_a x_{a,i} B_{a,j} defines the shape-function gradients
B (B_a = row a-1 of D_m^{-1} for a >= 1, B_0 = -sum_a B_a).

The constraint of Eq. optProb is c(x, p) = dPi/dx with the potential
Pi = sum_e vol_e Psi(F_e) - f_ext . x, so dc/dx is the assembled Hessian and
dc/dp_e is the force of element e alone (Psi is linear in E, E = E0 e^p).
"""
from __future__ import annotations

import numpy as np


def lame(E, nu):
    """Lame constants of Young's modulus E (array) and Poisson ratio nu."""
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def rest_geometry(X, conn):
    """D_m^{-1} (n_e, d, d), rest volumes (n_e,), B (n_e, d+1, d)."""
    d = X.shape[1]
    Dm = np.stack([X[conn[:, a]] - X[conn[:, 0]] for a in range(1, d + 1)], axis=2)
    detDm = np.linalg.det(Dm)
    vol = np.abs(detDm) / (2.0 if d == 2 else 6.0)
    Dminv = np.linalg.inv(Dm)
    B = np.empty((conn.shape[0], d + 1, d), dtype=np.float64)
    B[:, 1:, :] = Dminv
    B[:, 0, :] = -Dminv.sum(axis=1)
    return Dminv, vol, B


def deformation_gradient(x, conn, Dminv):
    """F = D_s D_m^{-1} for every element; x may be complex."""
    d = Dminv.shape[1]
    Ds = np.stack([x[conn[:, a]] - x[conn[:, 0]] for a in range(1, d + 1)], axis=2)
    return Ds @ Dminv


def deformation_gradient_disp(u, conn, Dminv):
    """F = I + D_u D_m^{-1} from node displacements u (x = X + u)."""
    d = Dminv.shape[1]
    Du = np.stack([u[conn[:, a]] - u[conn[:, 0]] for a in range(1, d + 1)], axis=2)
    return np.eye(d)[None] + Du @ Dminv


def _F(x, u, conn, Dminv):
    return deformation_gradient(x, conn, Dminv) if u is None else deformation_gradient_disp(u, conn, Dminv)


def energy_density(F, mu, lam):
    d = F.shape[1]
    J = np.linalg.det(F)
    lnJ = np.log(J)
    I1 = np.einsum("eij,eij->e", F, F)
    return 0.5 * mu * (I1 - d) - mu * lnJ + 0.5 * lam * lnJ * lnJ


def first_piola(F, mu, lam):
    """P = dPsi/dF = mu (F - F^{-T}) + lambda ln J F^{-T}."""
    J = np.linalg.det(F)
    FinvT = np.transpose(np.linalg.inv(F), (0, 2, 1))
    lnJ = np.log(J)
    return mu[:, None, None] * (F - FinvT) + (lam * lnJ)[:, None, None] * FinvT


def piola_tangent(F, mu, lam):
    """dP_ij/dF_kl as an (n_e, d, d, d, d) array:
    mu d_ik d_jl + (mu - lambda ln J) Finv_jk Finv_li + lambda Finv_ji Finv_lk."""
    d = F.shape[1]
    Finv = np.linalg.inv(F)
    lnJ = np.log(np.linalg.det(F))
    eye = np.eye(d)
    T = mu[:, None, None, None, None] * np.einsum("ik,jl->ijkl", eye, eye)[None]
    T = T + (mu - lam * lnJ)[:, None, None, None, None] * np.einsum("ejk,eli->eijkl", Finv, Finv)
    T = T + lam[:, None, None, None, None] * np.einsum("eji,elk->eijkl", Finv, Finv)
    return T


def element_energy(x, X, conn, E, nu, u=None):
    """vol_e Psi(F_e) per element (positions x, or displacements u)."""
    Dminv, vol, _ = rest_geometry(X, conn)
    F = _F(x, u, conn, Dminv)
    mu, lam = lame(E, nu)
    return vol * energy_density(F, mu, lam)


def element_force(x, X, conn, E, nu, u=None):
    """Gradient of vol Psi w.r.t. the element's node positions,
    (n_e, d+1, d): f_{a,k} = vol sum_j P_kj B_aj."""
    _, vol, B = rest_geometry(X, conn)
    Dminv = B[:, 1:, :]
    F = _F(x, u, conn, Dminv)
    mu, lam = lame(E, nu)
    P = first_piola(F, mu, lam)
    return vol[:, None, None] * np.einsum("ekj,eaj->eak", P, B)


def element_hessian(x, X, conn, E, nu, u=None):
    """Hessian of vol Psi w.r.t. the element's node positions,
    (n_e, d+1, d, d+1, d): K[a,m,b,n] = vol sum_jl B_aj dP_mj/dF_nl B_bl."""
    _, vol, B = rest_geometry(X, conn)
    Dminv = B[:, 1:, :]
    F = _F(x, u, conn, Dminv)
    mu, lam = lame(E, nu)
    T = piola_tangent(F, mu, lam)
    return vol[:, None, None, None, None] * np.einsum("eaj,emjnl,ebl->eambn", B, T, B)


def element_jacobian_det(x, X, conn, u=None):
    Dminv, _, _ = rest_geometry(X, conn)
    return np.linalg.det(_F(x, u, conn, Dminv))
