"""Pins of the oracle's element model (complex-step derivatives, the
linear-elastic closed form at F = I, frame indifference, a uniform-stretch
closed form, and the parameter column)."""
import numpy as np
import pytest

from oracle import elements as el
from sgn_inputs import grid2d, kuhn3d


def _disconnected(d, n_el, seed, strain=0.15):
    """n_el independent random simplices (own nodes) with random deformed
    positions near the rest shape."""
    rng = np.random.default_rng(seed)
    if d == 2:
        X0, c0 = grid2d(3)
    else:
        X0, c0 = kuhn3d(3)
    c0 = c0[rng.integers(0, c0.shape[0], size=n_el)]
    X = X0[c0].reshape(-1, d) + 0.01 * rng.standard_normal((n_el * (d + 1), d))
    conn = np.arange(n_el * (d + 1), dtype=np.int32).reshape(n_el, d + 1)
    x = X + strain * 0.2 * rng.standard_normal(X.shape)
    E = 1e4 * np.exp(rng.normal(0.0, 0.3, size=n_el))
    return X, conn, x, E


@pytest.mark.parametrize("d", [2, 3])
def test_force_is_complex_step_gradient_of_energy(d):
    X, conn, x, E = _disconnected(d, 64, seed=d)
    f = el.element_force(x, X, conn, E, 0.3)
    h = 1e-30
    for a in range(d + 1):
        for k in range(d):
            xc = x.astype(np.complex128)
            xc[conn[:, a], k] += 1j * h
            g = np.imag(el.element_energy(xc, X, conn, E, 0.3)) / h
            np.testing.assert_allclose(f[:, a, k], g, rtol=1e-12, atol=1e-12 * np.abs(f).max())


@pytest.mark.parametrize("d", [2, 3])
def test_hessian_is_complex_step_jacobian_of_force(d):
    X, conn, x, E = _disconnected(d, 64, seed=10 + d)
    H = el.element_hessian(x, X, conn, E, 0.3)
    h = 1e-30
    for b in range(d + 1):
        for n in range(d):
            xc = x.astype(np.complex128)
            xc[conn[:, b], n] += 1j * h
            col = np.imag(el.element_force(xc, X, conn, E, 0.3)) / h
            np.testing.assert_allclose(H[:, :, :, b, n], col, rtol=1e-11,
                                       atol=1e-12 * np.abs(H).max())
    # symmetry of the element Hessian
    nd = (d + 1) * d
    Hm = H.reshape(-1, nd, nd)
    np.testing.assert_allclose(Hm, np.transpose(Hm, (0, 2, 1)), rtol=0, atol=1e-12 * np.abs(Hm).max())


def _linear_elastic_stiffness(X, conn, E, nu):
    """Classical small-strain stiffness vol * Bv^T Dmat Bv (Voigt notation,
    engineering shear strains), with the shape-function gradients taken from
    the inverse of the barycentric-coordinate matrix [1 X^T]."""
    d = X.shape[1]
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    out = []
    for e in range(conn.shape[0]):
        Xe = X[conn[e]]
        Mb = np.hstack([np.ones((d + 1, 1)), Xe])
        coef = np.linalg.inv(Mb)            # column a: coefficients of N_a
        grad = coef[1:, :].T                 # (d+1, d): dN_a/dX_j
        vol = abs(np.linalg.det(Mb)) / (2.0 if d == 2 else 6.0)
        if d == 2:
            Bv = np.zeros((3, 6))
            for a in range(3):
                Bv[0, 2 * a] = grad[a, 0]
                Bv[1, 2 * a + 1] = grad[a, 1]
                Bv[2, 2 * a] = grad[a, 1]
                Bv[2, 2 * a + 1] = grad[a, 0]
            D = np.array([[lam[e] + 2 * mu[e], lam[e], 0], [lam[e], lam[e] + 2 * mu[e], 0],
                          [0, 0, mu[e]]])
        else:
            Bv = np.zeros((6, 12))
            for a in range(4):
                gx, gy, gz = grad[a]
                c = 3 * a
                Bv[0, c] = gx; Bv[1, c + 1] = gy; Bv[2, c + 2] = gz
                Bv[3, c] = gy; Bv[3, c + 1] = gx
                Bv[4, c + 1] = gz; Bv[4, c + 2] = gy
                Bv[5, c] = gz; Bv[5, c + 2] = gx
            D = np.zeros((6, 6))
            D[:3, :3] = lam[e]
            D[np.arange(3), np.arange(3)] += 2 * mu[e]
            D[3:, 3:] = np.eye(3) * mu[e]
        out.append(vol * Bv.T @ D @ Bv)
    return np.array(out)


@pytest.mark.parametrize("d", [2, 3])
def test_hessian_at_rest_is_linear_elastic_stiffness(d):
    X, conn, _, E = _disconnected(d, 20, seed=20 + d)
    H = el.element_hessian(X.copy(), X, conn, E, 0.3)
    nd = (d + 1) * d
    Klin = _linear_elastic_stiffness(X, conn, E, 0.3)
    np.testing.assert_allclose(H.reshape(-1, nd, nd), Klin, rtol=1e-11, atol=1e-9 * np.abs(Klin).max())


def _rotation(d, rng):
    Q, R = np.linalg.qr(rng.standard_normal((d, d)))
    Q = Q * np.sign(np.diag(R))[None, :]
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


@pytest.mark.parametrize("d", [2, 3])
def test_rigid_motion_is_stress_free_and_frame_indifferent(d):
    rng = np.random.default_rng(30 + d)
    X, conn, x, E = _disconnected(d, 32, seed=30 + d)
    R = _rotation(d, rng)
    t = rng.standard_normal(d)
    xr = X @ R.T + t
    assert np.max(np.abs(el.element_energy(xr, X, conn, E, 0.3))) < 1e-9
    f = el.element_force(xr, X, conn, E, 0.3)
    assert np.max(np.abs(f)) < 1e-9 * E.max()
    # f(R x + t) = R f(x) and energy invariant, for a deformed x
    f0 = el.element_force(x, X, conn, E, 0.3)
    f1 = el.element_force(x @ R.T + t, X, conn, E, 0.3)
    np.testing.assert_allclose(f1, f0 @ R.T, rtol=1e-10, atol=1e-10 * np.abs(f0).max())
    np.testing.assert_allclose(el.element_energy(x @ R.T + t, X, conn, E, 0.3),
                               el.element_energy(x, X, conn, E, 0.3), rtol=1e-10)


@pytest.mark.parametrize("d,n", [(2, 5), (3, 4)])
def test_uniform_stretch_energy_closed_form(d, n):
    """x = diag(s,1,..) X: every element has F = diag(s, 1, ...), so the total
    energy is |Omega| (mu/2 (s^2-1) - mu ln s + lambda/2 ln^2 s) with
    |Omega| = 1 for the unit square / cube."""
    X, conn = grid2d(n) if d == 2 else kuhn3d(n)
    s = 1.3
    x = X.copy()
    x[:, 0] *= s
    E0, nu = 2.5e3, 0.3
    E = np.full(conn.shape[0], E0)
    mu = E0 / (2 * (1 + nu))
    lam = E0 * nu / ((1 + nu) * (1 - 2 * nu))
    want = mu / 2 * (s * s - 1) - mu * np.log(s) + lam / 2 * np.log(s) ** 2
    got = el.element_energy(x, X, conn, E, nu).sum()
    assert abs(got - want) < 1e-12 * abs(want)


@pytest.mark.parametrize("d", [2, 3])
def test_parameter_column_is_complex_step_in_p(d):
    """dc/dp_e equals the force of element e (E = E0 e^p)."""
    X, conn, x, _ = _disconnected(d, 16, seed=40 + d)
    rng = np.random.default_rng(41)
    p = rng.normal(0.0, 0.2, size=conn.shape[0])
    h = 1e-30
    f = el.element_force(x, X, conn, 1e4 * np.exp(p), 0.3)
    fc = el.element_force(x.astype(np.complex128), X, conn, 1e4 * np.exp(p + 1j * h), 0.3)
    np.testing.assert_allclose(np.imag(fc) / h, f, rtol=1e-12, atol=1e-14 * np.abs(f).max())


def test_planted_mistake_is_caught(monkeypatch):
    """Dropping the lambda term of dP/dF must break the complex-step pin."""
    orig = el.piola_tangent

    def broken(F, mu, lam):
        return orig(F, mu, 0.0 * lam) + 0.0 * lam[:, None, None, None, None]

    monkeypatch.setattr(el, "piola_tangent", broken)
    with pytest.raises(AssertionError):
        test_hessian_is_complex_step_jacobian_of_force(3)


@pytest.mark.parametrize("d", [2, 3])
def test_displacement_form_equals_position_form(d):
    """F = I + D_u D_m^{-1} (u = x - X) is D_s D_m^{-1} rewritten: the two
    agree to rounding, and at u = 0 the displacement form is I exactly, so
    the energy and the force vanish exactly at rest."""
    X, conn, x, E = _disconnected(d, 64, seed=10 + d)
    u = x - X
    f_pos = el.element_force(x, X, conn, E, 0.3)
    f_dis = el.element_force(None, X, conn, E, 0.3, u=u)
    np.testing.assert_allclose(f_dis, f_pos, rtol=0, atol=1e-10 * np.abs(f_pos).max())
    H_pos = el.element_hessian(x, X, conn, E, 0.3)
    H_dis = el.element_hessian(None, X, conn, E, 0.3, u=u)
    np.testing.assert_allclose(H_dis, H_pos, rtol=0, atol=1e-10 * np.abs(H_pos).max())
    z = np.zeros_like(X)
    assert np.all(el.element_energy(None, X, conn, E, 0.3, u=z) == 0.0)
    assert np.all(el.element_force(None, X, conn, E, 0.3, u=z) == 0.0)
    Dminv, _, _ = el.rest_geometry(X, conn)
    assert np.all(el.deformation_gradient_disp(z, conn, Dminv) == np.eye(d)[None])
