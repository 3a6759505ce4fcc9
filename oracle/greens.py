"""Fourier transforms of the truncated free-space Green's functions (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 5 (numerical results) applies the volume potentials of Eqs. (Vo) and (Vw)
by (a) truncating the Green's function to the range of interest, (b) taking the
Fourier transform of the truncated kernel, a smooth function, and (c) cutting
it off at the grid's Nyquist frequency.  Step (b) has a closed form.  With the
transform convention ``f^(k) = int f(x) exp(-i k.x) dx`` and ``kappa = |k|``:

    G_L(x) = exp(i w |x|) / (4 pi |x|)  for |x| <= L, else 0
    G^_L(kappa) = (1/kappa) int_0^L sin(kappa r) exp(i w r) dr        (radial transform)

For ``w = 0`` (Laplace, Eq. (Vo)) this is ``2 sin^2(L kappa / 2) / kappa^2``.

Evaluation (stable everywhere, no cancellation at kappa = w):
    sin(kappa r) = (e^{i kappa r} - e^{-i kappa r}) / 2i  gives
    G^_L(kappa) = [E(w + kappa) - E(w - kappa)] / (2 i kappa),
    E(a) = int_0^L e^{i a r} dr = L exp(i a L / 2) sinc(a L / 2),  sinc(t) = sin(t)/t.
E is entire and evaluated without cancellation for every real a, so the
apparent singularity of the textbook closed form at kappa = w is gone.  The
difference of two E values loses accuracy only as kappa L -> 0; there
(kappa L < 0.05, which on the grids used here means kappa = 0 only) the
defining integral ``int_0^L r sinc(kappa r) exp(i w r) dr`` is evaluated by
Gauss-Legendre quadrature with enough nodes to integrate it to rounding.
"""
from __future__ import annotations

import numpy as np

SMALL_KAPPA_L = 0.05


def _sinc(t):
    t = np.asarray(t, dtype=np.float64)
    out = np.ones_like(t)
    nz = t != 0.0
    out[nz] = np.sin(t[nz]) / t[nz]
    return out


def _E(a, L):
    """int_0^L exp(i a r) dr for real a (vectorised)."""
    return L * np.exp(0.5j * a * L) * _sinc(0.5 * a * L)


def _quad_small_kappa(kappa, omega, L):
    """int_0^L r sinc(kappa r) e^{i w r} dr by Gauss-Legendre (entire integrand)."""
    kappa = np.atleast_1d(np.asarray(kappa, dtype=np.float64))
    nodes = int(64 + (abs(omega) + float(np.max(kappa, initial=0.0))) * L)
    t, w = np.polynomial.legendre.leggauss(nodes)
    r = 0.5 * L * (t + 1.0)
    wt = 0.5 * L * w
    vals = (r[None, :] * _sinc(kappa[:, None] * r[None, :]) * np.exp(1j * omega * r)[None, :]) @ wt
    return vals


def truncated_green_hat(kappa, omega: float, L: float):
    """G^_L(kappa) for the truncated kernel exp(i w r)/(4 pi r), r <= L (Sec. 5, steps a-b).

    ``kappa`` may be an array (>= 0).  ``omega = 0`` gives the Laplace kernel of Eq. (Vo).
    Returns complex128 with the shape of ``kappa``.
    """
    kappa = np.asarray(kappa, dtype=np.float64)
    shape = kappa.shape
    kf = kappa.ravel()
    out = np.empty(kf.shape, np.complex128)
    small = kf * L < SMALL_KAPPA_L
    big = ~small
    if np.any(big):
        k = kf[big]
        out[big] = (_E(omega + k, L) - _E(omega - k, L)) / (2j * k)
    if np.any(small):
        out[small] = _quad_small_kappa(kf[small], omega, L)
    return out.reshape(shape)

