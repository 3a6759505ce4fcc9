"""Linear solvers for (I+B+K) J = b (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``neumann``: J = sum_n (I - A)^n b, the series of the existence proof of
  Sec. 2 (converges because ||B|| < 1, Lemmas 1-2).
* ``gmres``: textbook restarted GMRES (Saad and Schultz 1986) with modified
  Gram-Schmidt Arnoldi and Givens rotations, float64/complex128 throughout.
  GMRES is named as applicable in Sec. 1 and Sec. 6.
* ``bicgstab``: van der Vorst's Bi-CGStab (1992), the solver of Sec. 5.
* ``dense_solve``: the matrix of the operator assembled column by column and
  solved by LU with partial pivoting (numpy.linalg.solve); tiny grids only.
"""
from __future__ import annotations

import numpy as np


def _dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def _nrm(a):
    return float(np.linalg.norm(a.ravel()))


def neumann(apply, b, tol=1e-13, maxiter=500):
    """Fixed point J <- b + (J - A J), i.e. the partial sums of sum_n B^n b."""
    x = b.copy()
    nb = _nrm(b)
    hist = []
    for it in range(maxiter):
        r = b - apply(x)
        rel = _nrm(r) / nb
        hist.append(rel)
        if rel <= tol:
            return x, {"iters": it, "residuals": hist, "converged": True}
        x = x + r
    return x, {"iters": maxiter, "residuals": hist, "converged": False}


def gmres(apply, b, x0=None, tol=1e-13, restart=50, maxiter=2000):
    """Restarted GMRES(m); stops when ||b - A x|| / ||b|| <= tol (true residual checked at restarts)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    nb = _nrm(b)
    hist = []
    total = 0
    while total < maxiter:
        r = b - apply(x)
        beta = _nrm(r)
        hist.append(beta / nb)
        if beta / nb <= tol:
            return x, {"iters": total, "residuals": hist, "converged": True}
        m = restart
        V = [r / beta]
        Hm = np.zeros((m + 1, m), np.complex128)
        cs = np.zeros(m, np.complex128)
        sn = np.zeros(m, np.complex128)
        g = np.zeros(m + 1, np.complex128)
        g[0] = beta
        j_done = 0
        for j in range(m):
            w = apply(V[j])
            total += 1
            for i in range(j + 1):
                Hm[i, j] = _dot(V[i], w)
                w = w - Hm[i, j] * V[i]
            hnorm = _nrm(w)
            Hm[j + 1, j] = hnorm
            # earlier rotations G_i = [[conj(c_i), conj(s_i)], [-s_i, c_i]] on rows i, i+1
            for i in range(j):
                t = np.conj(cs[i]) * Hm[i, j] + np.conj(sn[i]) * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            a, bb = Hm[j, j], Hm[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[j] = a / den if den != 0 else 1.0
            sn[j] = bb / den if den != 0 else 0.0
            Hm[j, j] = np.conj(cs[j]) * a + np.conj(sn[j]) * bb
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            j_done = j + 1
            if abs(g[j + 1]) / nb <= tol * 0.5 or hnorm == 0.0 or total >= maxiter:
                break
            if j + 1 < m:
                V.append(w / _nrm(w))
        y = np.linalg.solve(np.triu(Hm[:j_done, :j_done]), g[:j_done])
        for i in range(j_done):
            x = x + y[i] * V[i]
    r = b - apply(x)
    hist.append(_nrm(r) / nb)
    return x, {"iters": total, "residuals": hist, "converged": hist[-1] <= tol}


def bicgstab(apply, b, x0=None, tol=1e-13, maxiter=2000):
    """Unpreconditioned Bi-CGStab (van der Vorst 1992); counts operator applies."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    nb = _nrm(b)
    r = b - apply(x)
    applies = 1 if x0 is not None else 0
    rhat = r.copy()
    rho = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    hist = [_nrm(r) / nb]
    for it in range(maxiter):
        rho_new = _dot(rhat, r)
        beta = (rho_new / rho) * (alpha / omega)
        rho = rho_new
        p = r + beta * (p - omega * v)
        v = apply(p)
        applies += 1
        alpha = rho / _dot(rhat, v)
        s = r - alpha * v
        if _nrm(s) / nb <= tol:
            x = x + alpha * p
            hist.append(_nrm(s) / nb)
            return x, {"iters": it + 1, "applies": applies, "residuals": hist, "converged": True}
        t = apply(s)
        applies += 1
        omega = _dot(t, s) / _dot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        hist.append(_nrm(r) / nb)
        if hist[-1] <= tol:
            return x, {"iters": it + 1, "applies": applies, "residuals": hist, "converged": True}
    return x, {"iters": maxiter, "applies": applies, "residuals": hist, "converged": False}


def assemble(apply, shape) -> np.ndarray:
    """Dense matrix of a linear operator on arrays of ``shape`` (column j = A e_j)."""
    size = int(np.prod(shape))
    A = np.empty((size, size), np.complex128)
    e = np.zeros(size, np.complex128)
    for j in range(size):
        e[j] = 1.0
        A[:, j] = apply(e.reshape(shape)).ravel()
        e[j] = 0.0
    return A


def dense_solve(apply, b) -> np.ndarray:
    """LU with partial pivoting on the assembled operator (numpy.linalg.solve)."""
    A = assemble(apply, b.shape)
    return np.linalg.solve(A, b.ravel()).reshape(b.shape)
