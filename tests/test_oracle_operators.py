"""Pins for the oracle's operators, right-hand sides, solvers and scattered fields.

* Lemma 1: ||H_eps(x)||_2 < 1 for real SPD eps; H = U f(D) U^T with f(z) = (z-1)/(z+1).
* H_{eps^-1} = -H_eps (used to relate Eqs. (eq:intLap) and (eq:intH)).
* Neumann series (Sec. 2 existence proof) = GMRES = Bi-CGStab = dense LU.
* Helmholtz at w -> 0 with eps equals Laplace with eps^-1 (same derivation).
* Maxwell: mu = I gives M = 0 and the reduced equation; w -> 0 reduces to
  Laplace with E_in = grad phi_in; the eps <-> mu, J -> M, M -> -J duality.
* Low-frequency stability of the J = J_V/(-iw) scaling (Tables 2-5: the
  1e-50 and 1e-10 wavelength rows agree).
* Smooth dielectric sphere (isotropic radial eps(r)): the grid solution J
  equals (eps - 1) grad phi, phi = f(r) cos(theta) from the radial ODE
  (r^2 eps f')' = 2 eps f solved to 1e-12 in 1D -- spectral convergence.
* Sharpening sphere: interior field tends to 3 E0 / (eps + 2).
* Lossless media: optical theorem int |A|^2 = (4 pi / w) Im A(d);
  reciprocity A(xhat; d) = A(-d; -xhat).
"""
import math

import numpy as np
import pytest
import scipy.special as sp
from scipy.integrate import solve_ivp

import vie_inputs as vi
from oracle import operators, solvers


def nrm(a):
    return float(np.linalg.norm(np.asarray(a).ravel()))


def test_lemma1_contraction_and_spectral_form():
    p = vi.laplace_bump_problem(n=8)
    H = operators.h_tensor(p.eps)
    Hm = np.moveaxis(H, (0, 1), (-2, -1)).reshape(-1, 3, 3)
    norms = np.linalg.norm(Hm, ord=2, axis=(-2, -1))
    assert norms.max() < 1.0
    E = np.moveaxis(p.eps, (0, 1), (-2, -1)).reshape(-1, 3, 3).real
    lam, U = np.linalg.eigh(E)
    f = (lam - 1) / (lam + 1)
    ref = np.einsum("pab,pb,pcb->pac", U, f, U)
    assert np.max(np.abs(Hm - ref)) <= 1e-14
    assert np.max(np.abs(Hm - np.swapaxes(Hm, -1, -2))) <= 1e-15
    for name in ("eps234", "eps_dense", "eps444"):
        eps = vi.paper_medium(name, 8)
        Hd = np.moveaxis(operators.h_tensor(eps), (0, 1), (-2, -1)).reshape(-1, 3, 3)
        assert np.linalg.norm(Hd, ord=2, axis=(-2, -1)).max() < 1.0


def test_h_of_inverse_is_minus_h():
    p = vi.helmholtz_problem(n=6, wavelengths=2.0)
    He = operators.h_tensor(p.eps)
    Hi = operators.h_tensor(operators.inverse_field(p.eps))
    assert np.max(np.abs(Hi + He)) <= 1e-14


def test_isotropic_h_closed_form():
    n = 4
    e = 2.5 + 0.3j
    eps = np.zeros((3, 3, n, n, n), np.complex128)
    for a in range(3):
        eps[a, a] = e
    H = operators.h_tensor(eps)
    for a in range(3):
        for b in range(3):
            assert np.allclose(H[a, b], (e - 1) / (e + 1) if a == b else 0.0, atol=1e-15)


def test_laplace_solvers_agree_with_dense_lu():
    p = vi.laplace_bump_problem(n=6)
    op = operators.OracleProblem.from_problem(p)
    b = op.rhs(p.directions[0])
    x_lu = solvers.dense_solve(op.apply, b)
    x_n, info = solvers.neumann(op.apply, b, tol=1e-14)
    assert info["converged"]
    x_g, ig = solvers.gmres(op.apply, b, tol=1e-14, restart=20)
    x_b, ib = solvers.bicgstab(op.apply, b, tol=1e-14)
    for x in (x_n, x_g, x_b):
        assert nrm(x - x_lu) <= 1e-12 * nrm(x_lu)


def test_helmholtz_solvers_agree_with_dense_lu():
    p = vi.helmholtz_problem(n=6, wavelengths=2.0)
    op = operators.OracleProblem.from_problem(p)
    b = op.rhs(p.directions[0])
    x_lu = solvers.dense_solve(op.apply, b)
    x_g, ig = solvers.gmres(op.apply, b, tol=1e-14, restart=15)
    assert ig["converged"]
    assert nrm(x_g - x_lu) <= 1e-12 * nrm(x_lu)
    assert nrm(op.apply(x_lu) - b) <= 1e-13 * nrm(b)


def test_helmholtz_low_frequency_is_laplace_with_inverse_eps():
    n = 8
    ph = vi.helmholtz_problem(n=n, wavelengths=1e-10)
    oh = operators.OracleProblem.from_problem(ph)
    ol = operators.OracleProblem("laplace", n, -1.0, 1.0, 0.0, operators.inverse_field(ph.eps))
    x = vi.random_field(n, 3, 5)[0]
    assert nrm(oh.apply(x) - ol.apply(x)) <= 1e-12 * nrm(ol.apply(x))


def test_maxwell_mu_identity_reduces():
    n = 6
    pm = vi.maxwell_problem(n=n, wavelengths=1.5, with_mu=False)
    red = operators.OracleProblem.from_problem(pm)
    mu_I = vi.identity_field(n)
    full = operators.OracleProblem("maxwell", n, -1.0, 1.0, pm.omega, pm.eps, mu_I)
    assert np.max(np.abs(full.Hmu)) == 0.0
    d, pol = pm.directions[0], pm.polarisations[0]
    b6 = full.rhs(d, pol)
    assert np.max(np.abs(b6[3:])) == 0.0
    x6, i6 = solvers.gmres(full.apply, b6, tol=1e-13, restart=30)
    x3, i3 = solvers.gmres(red.apply, red.rhs(d, pol), tol=1e-13, restart=30)
    assert nrm(x6[3:]) <= 1e-12 * nrm(x6)
    assert nrm(x6[:3] - x3) <= 1e-11 * nrm(x3)


@pytest.mark.parametrize("kind", ["laplace", "helmholtz", "maxwell"])
def test_vacuum_operator_is_identity(kind):
    """No scatterer (eps = mu = I): H = 0 (Eq. (rhodef)), so B and K vanish and the
    operator is exactly the identity; the right-hand side is zero and so is J."""
    n = 6
    eye = vi.identity_field(n)
    op = operators.OracleProblem(kind, n, -1.0, 1.0, 0.0 if kind == "laplace" else 2.0, eye,
                                 eye if kind == "maxwell" else None)
    x = vi.random_field(n, op.ncomp, 11)[0]
    assert np.array_equal(op.apply(x), x)
    b = op.rhs(np.array([0.0, 0.6, 0.8]), np.array([1.0, 0.0, 0.0]) if kind == "maxwell" else None)
    assert np.max(np.abs(b)) == 0.0


def test_maxwell_low_frequency_is_laplace():
    n = 6
    pm = vi.maxwell_problem(n=n, wavelengths=1e-10, with_mu=False)
    om = operators.OracleProblem.from_problem(pm)
    ol = operators.OracleProblem("laplace", n, -1.0, 1.0, 0.0, pm.eps)
    x = vi.random_field(n, 3, 7)[0]
    assert nrm(om.apply(x) - ol.apply(x)) <= 1e-12 * nrm(ol.apply(x))


def test_maxwell_duality():
    n = 6
    pm = vi.maxwell_problem(n=n, wavelengths=2.0)
    a = operators.OracleProblem("maxwell", n, -1.0, 1.0, pm.omega, pm.eps, pm.mu)
    b = operators.OracleProblem("maxwell", n, -1.0, 1.0, pm.omega, pm.mu, pm.eps)
    x = vi.random_field(n, 6, 11)[0]
    ya = a.apply(x)
    yb = b.apply(np.concatenate([x[3:], -x[:3]]))
    assert nrm(yb - np.concatenate([ya[3:], -ya[:3]])) <= 1e-13 * nrm(ya)


def test_maxwell_low_frequency_stability():
    """J = J_V/(-iw) keeps the system regular: solutions at 1e-10 and 1e-50 wavelengths agree."""
    n = 6
    sols = []
    for wl in (1e-10, 1e-50):
        pm = vi.maxwell_problem(n=n, wavelengths=wl, with_mu=True)
        op = operators.OracleProblem.from_problem(pm)
        b = op.rhs(pm.directions[0], pm.polarisations[0])
        x, info = solvers.gmres(op.apply, b, tol=1e-14, restart=40)
        assert info["converged"]
        sols.append(x)
    assert nrm(sols[0] - sols[1]) <= 1e-10 * nrm(sols[1])


# ------------------------------------------------------------ sphere pins


def radial_sphere_solution(eps_r, Rmax=1.0):
    """phi = f(r) cos(theta) for div(eps grad phi) = 0, f -> -r at infinity, regular at 0.

    (r^2 eps f')' = 2 eps f; integrate q = r^2 eps f' and f from r0 with f = r, then
    match f = A r + B / r^2 outside the medium and scale so that A = -1.
    """
    r0 = 1e-6

    def rhs(r, y):
        f, q = y
        e = eps_r(r)
        return [q / (r * r * e), 2.0 * e * f]

    y0 = [r0, r0 * r0 * eps_r(r0)]
    sol = solve_ivp(rhs, (r0, Rmax), y0, method="DOP853", rtol=1e-13, atol=1e-16, dense_output=True)
    fR, qR = sol.y[:, -1]
    fpR = qR / (Rmax * Rmax * eps_r(Rmax))
    # f = A r + B r^-2, f' = A - 2 B r^-3
    A = (2.0 * fR / Rmax + fpR) / 3.0
    scale = -1.0 / A

    def f_and_fp(r):
        y = sol.sol(r)
        return scale * y[0], scale * y[1] / (r * r * eps_r(r))

    return f_and_fp


def test_smooth_sphere_matches_radial_ode():
    R0, delta, eps_s = 0.4, 0.12, 3.0
    eps_r = lambda r: 1.0 + (eps_s - 1.0) * 0.5 * sp.erfc((r - R0) / delta)
    f_fp = radial_sphere_solution(eps_r)
    errs = []
    for n in (24, 40):
        eps = vi.smooth_sphere_eps(n, eps_s, R0, delta)
        op = operators.OracleProblem("laplace", n, -1.0, 1.0, 0.0, eps)
        b = op.rhs([0.0, 0.0, 1.0])
        J, info = solvers.gmres(op.apply, b, tol=1e-12, restart=40)
        Z, Y, X = op.grid.coords()
        r = np.sqrt(X * X + Y * Y + Z * Z) + 0 * X
        fr, fpr = f_fp(np.clip(r.ravel(), 1e-6, 1.0))
        fr, fpr = fr.reshape(r.shape), fpr.reshape(r.shape)
        zr = Z / r
        rad = (fpr - fr / r) * zr
        grad = np.stack([rad * X / r, rad * Y / r, rad * Z / r + fr / r])
        e1 = 1.0 + (eps_s - 1.0) * 0.5 * sp.erfc((r - R0) / delta)
        Jref = (e1 - 1.0) * grad
        errs.append(nrm(J - Jref) / nrm(Jref))
    assert errs[1] < 1e-5 and errs[1] < errs[0] / 20


def test_sharpening_sphere_interior_field():
    """Homogeneous sphere limit: interior E -> 3 E0/(eps + 2) as the profile sharpens (O(delta))."""
    eps_s = 3.0
    vals = []
    for n, delta in ((24, 0.12), (40, 0.06)):
        eps = vi.smooth_sphere_eps(n, eps_s, 0.5, delta)
        op = operators.OracleProblem("laplace", n, -1.0, 1.0, 0.0, eps)
        J, _ = solvers.gmres(op.apply, op.rhs([0.0, 0.0, 1.0]), tol=1e-10, restart=40)
        c = n // 2
        Ez = -J[2, c - 1:c + 1, c - 1:c + 1, c - 1:c + 1].real.mean() / (eps_s - 1.0)
        vals.append(Ez)
    target = 3.0 / (eps_s + 2.0)
    assert abs(vals[1] - target) < abs(vals[0] - target)
    assert abs(vals[1] - target) < 0.03


# ----------------------------------------------- energy and reciprocity


def far_field_amplitude(op, J, xhat):
    """A(xhat) = i w xhat . J^(w xhat) / (4 pi), J^(k) = h^3 sum_j J_j exp(-i k . y_j)."""
    g = op.grid
    Z, Y, X = g.coords()
    w = op.omega
    out = []
    for u in xhat:
        ph = np.exp(-1j * w * (u[0] * X + u[1] * Y + u[2] * Z)) * g.h ** 3
        Jh = np.array([np.sum(J[a] * ph) for a in range(3)])
        out.append(1j * w * (u @ Jh) / (4 * np.pi))
    return np.array(out)


def sphere_quadrature(nt=24, nph=48):
    t, wt = np.polynomial.legendre.leggauss(nt)
    ph = 2 * np.pi * np.arange(nph) / nph
    ct = np.repeat(t, nph)
    st = np.sqrt(1 - ct * ct)
    p = np.tile(ph, nt)
    dirs = np.stack([st * np.cos(p), st * np.sin(p), ct], -1)
    w = np.repeat(wt, nph) * (2 * np.pi / nph)
    return dirs, w


@pytest.fixture(scope="module")
def lossless_helmholtz():
    p = vi.helmholtz_problem(n=32, wavelengths=1.5, lossless=True, nrhs=2, seed=3)
    op = operators.OracleProblem.from_problem(p)
    sols = []
    for d in p.directions:
        J, info = solvers.gmres(op.apply, op.rhs(d), tol=1e-12, restart=60)
        assert info["converged"]
        sols.append(J)
    return p, op, sols


def test_optical_theorem_lossless(lossless_helmholtz):
    p, op, sols = lossless_helmholtz
    dirs, w = sphere_quadrature()
    d = p.directions[0]
    A = far_field_amplitude(op, sols[0], dirs)
    Ad = far_field_amplitude(op, sols[0], [d])[0]
    lhs = float(np.sum(w * np.abs(A) ** 2))
    rhs = 4 * np.pi / op.omega * Ad.imag
    assert abs(lhs - rhs) <= 1e-6 * abs(rhs)


def test_reciprocity(lossless_helmholtz):
    p, op, sols = lossless_helmholtz
    d1, d2 = p.directions
    a12 = far_field_amplitude(op, sols[0], [-d2])[0]  # A(-d2; d1)
    a21 = far_field_amplitude(op, sols[1], [-d1])[0]  # A(-d1; d2)
    assert abs(a12 - a21) <= 1e-8 * abs(a12)


def test_planted_helmholtz_sign_error_breaks_optical_theorem(lossless_helmholtz):
    """The printed '+2H' of Eq. (eq:intH) (a planted change, in the oracle) violates energy balance."""
    p, op, _ = lossless_helmholtz
    wrong = lambda x: x + 2.0 * operators.tmul(op.Hinv, operators.T_op(op.kt, x))
    J, info = solvers.gmres(wrong, op.rhs(p.directions[0]), tol=1e-10, restart=60, maxiter=400)
    dirs, w = sphere_quadrature()
    A = far_field_amplitude(op, J, dirs)
    Ad = far_field_amplitude(op, J, [p.directions[0]])[0]
    lhs = float(np.sum(w * np.abs(A) ** 2))
    rhs = 4 * np.pi / op.omega * Ad.imag
    assert abs(lhs - rhs) > 1e-3 * abs(rhs)
