"""Pins for the oracle's truncated Green's function transform (Sec. 5, steps a-b).

The oracle evaluates G^_L(kappa) = (1/kappa) int_0^L sin(kappa r) e^{i w r} dr by a
difference of two entire functions.  It is checked here against things it does
not share code with:
* mpmath adaptive quadrature (50 digits) of the radial Fourier integral
  int_0^L 4 pi r^2 G(r) sinc(kappa r) dr of the truncated kernel itself;
* the closed form of the truncated Laplace transform 2 sin^2(L kappa/2)/kappa^2;
* the kappa -> 0 and kappa -> w limits derived by hand
  (e^{iwL}(1 - iwL) - 1)/w^2 and i(L - e^{iwL} sin(wL)/w)/(2w).
"""
import math

import mpmath as mp
import numpy as np
import pytest

from oracle.greens import truncated_green_hat

mp.mp.dps = 50


def radial_transform_mp(kappa, omega, L):
    """int_0^L 4 pi r^2 [e^{i w r}/(4 pi r)] sinc(kappa r) dr with mpmath."""
    kappa = mp.mpf(kappa)
    omega = mp.mpf(omega)

    def f(r):
        s = mp.sin(kappa * r) / (kappa * r) if kappa != 0 else mp.mpf(1)
        return r * s * mp.expj(omega * r)

    pts = mp.linspace(0, L, 40)
    return complex(mp.quad(f, pts))


L = 2.0 * math.sqrt(3.0)


@pytest.mark.parametrize("omega", [0.0, 1e-9, 0.7, 4 * math.pi, 10 * math.pi])
@pytest.mark.parametrize("kappa", [0.0, 1e-6, 0.01, 1.0471975511965976, 3.3, 12.0, 57.3])
def test_against_quadrature(omega, kappa):
    ref = radial_transform_mp(kappa, omega, L)
    got = complex(truncated_green_hat(np.array([kappa]), omega, L)[0])
    # rounding floor: the integrand is bounded by L, so absolute errors of
    # order eps * L * min(L, 1/kappa) are unavoidable where the value cancels
    floor = 2e-14 * L * min(L, 1.0 / kappa if kappa > 0 else L)
    assert abs(got - ref) <= 1e-13 * abs(ref) + floor


@pytest.mark.parametrize("omega", [0.7, 4 * math.pi, 10 * math.pi])
@pytest.mark.parametrize("rel", [0.0, 1e-12, -1e-9, 1e-9, 1e-6, -1e-3])
def test_near_kappa_equals_omega(omega, rel):
    """kappa = w (1 + rel): the textbook closed form is 0/0 here; the oracle must not lose digits."""
    kappa = omega * (1.0 + rel)
    ref = radial_transform_mp(kappa, omega, L)
    got = complex(truncated_green_hat(np.array([kappa]), omega, L)[0])
    assert abs(got - ref) <= 1e-13 * abs(ref)


def test_kappa_equals_omega_closed_form():
    for omega in (0.3, 2.0, 4 * math.pi):
        ref = 1j * (L - np.exp(1j * omega * L) * math.sin(omega * L) / omega) / (2 * omega)
        got = truncated_green_hat(np.array([omega]), omega, L)[0]
        assert abs(got - ref) <= 1e-13 * abs(ref)


def test_kappa_zero_closed_form():
    for omega in (0.5, 3.0, 4 * math.pi):
        ref = (np.exp(1j * omega * L) * (1 - 1j * omega * L) - 1) / omega ** 2
        got = truncated_green_hat(np.array([0.0]), omega, L)[0]
        assert abs(got - ref) <= 1e-13 * abs(ref)


def test_laplace_closed_form():
    """w = 0: the transform of the truncated 1/(4 pi r) is 2 sin^2(L k/2)/k^2 (value L^2/2 at 0)."""
    kappa = np.concatenate([[0.0], np.linspace(1e-3, 300.0, 2001)])
    got = truncated_green_hat(kappa, 0.0, L)
    ref = np.empty_like(kappa)
    ref[0] = L * L / 2
    ref[1:] = 2 * np.sin(L * kappa[1:] / 2) ** 2 / kappa[1:] ** 2
    assert np.max(np.abs(got - ref)) <= 1e-13 * L * L / 2
    assert np.max(np.abs(got.imag)) == 0.0


def test_small_omega_limit_is_laplace():
    """w -> 0 (the 1e-50 / 1e-10 wavelength rows of Tables 2-5) recovers the Laplace transform.

    |e^{iwr} - 1| <= w r bounds the difference by w L^3 / 3.
    """
    kappa = np.linspace(0.0, 200.0, 1001)
    b = truncated_green_hat(kappa, 0.0, L)
    for omega in (2 * math.pi * 1e-10, 1e-6):
        a = truncated_green_hat(kappa, omega, L)
        assert np.max(np.abs(a - b)) <= omega * L ** 3 / 3 + 1e-14 * L * L
    a = truncated_green_hat(kappa, 2 * math.pi * 1e-50, L)
    assert np.max(np.abs(a - b)) <= 1e-14 * L * L
