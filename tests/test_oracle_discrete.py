"""Pins for the oracle's discrete convolution kernels (Sec. 5: truncate, transform, cut off).

* The FFT route equals the Fourier sum written out, and the (2n)^3 circular
  convolution equals the explicit Toeplitz product (brute force at 8^3).
* Kernel parity: -k_a k_b kernels are real for Laplace and odd/even in each axis.
* Newton potential of a Gaussian density: V_0 rho = erf(sqrt(a) r)/(4 pi r)
  (closed form), spectrally accurate once the Gaussian is resolved.
* Helmholtz potential of the same density, by the l = 0 addition theorem and
  1D quadrature (independent of any 3D machinery).
* Lemma 2: 2 T_0 grad psi = -grad psi and 2 T_w curl P = curl P.
* Delta V_0 rho = -rho (the identity stated after Eq. (Vo)).
"""
import math

import numpy as np
import pytest
import scipy.special as sp
from scipy import integrate

from oracle import discrete, operators

ALPHA = 36.0  # exp(-36) ~ 2e-16 at the faces of [-1,1]^3


def gaussian(grid):
    Z, Y, X = grid.coords()
    r2 = X * X + Y * Y + Z * Z
    return (ALPHA / np.pi) ** 1.5 * np.exp(-ALPHA * r2), np.sqrt(r2)


@pytest.mark.parametrize("n,omega", [(8, 0.0), (8, 3.7), (5, 3.7)])
def test_fft_kernels_equal_direct_sum(n, omega):
    g = discrete.Grid(n)
    src, dst, d = discrete._offset_indices(g)
    n = g.n
    for name in discrete.SYMBOLS:
        e = discrete.kernel_fft(name, g, omega)
        kd = discrete.kernel_direct(name, g, omega)
        a = e[np.ix_(dst, dst, dst)]
        b = kd[np.ix_(d + n - 1, d + n - 1, d + n - 1)]
        assert np.max(np.abs(a - b)) <= 1e-15 * max(1.0, np.max(np.abs(b))) * 10, name
        assert np.all(e[n, :, :] == 0) and np.all(e[:, n, :] == 0) and np.all(e[:, :, n] == 0)


def test_kernel_direct_single_term_loop():
    """One offset of one kernel by an explicit triple loop over the (sn)^3 frequencies."""
    g = discrete.Grid(4)
    sn = g.sn
    omega = 1.3
    kd = discrete.kernel_direct("xy", g, omega)
    from oracle.greens import truncated_green_hat

    d = (1, -2, 3)  # (dz, dy, dx)
    acc = 0j
    for mz in range(-sn // 2, sn // 2):
        for my in range(-sn // 2, sn // 2):
            for mx in range(-sn // 2, sn // 2):
                kz, ky, kx = (2 * np.pi * m / (3 * g.D) for m in (mz, my, mx))
                ox = 0.0 if mx == -sn // 2 else kx
                oy = 0.0 if my == -sn // 2 else ky
                kap = math.sqrt(kx * kx + ky * ky + kz * kz)
                G = truncated_green_hat(np.array([kap]), omega, g.L)[0]
                acc += -ox * oy * G * np.exp(2j * np.pi * (mz * d[0] + my * d[1] + mx * d[2]) / sn)
    acc /= sn ** 3
    got = kd[d[0] + 3, d[1] + 3, d[2] + 3]
    assert abs(got - acc) <= 1e-14 * max(1.0, abs(acc))


def test_kernel_direct_single_term_loop_odd_grid():
    """Odd n: the oversampled grid sn = 3n is odd, the cut set |m_a| <= (sn-1)/2 is
    symmetric and has no Nyquist entry, so every odd factor k_a is kept."""
    g = discrete.Grid(3)
    sn = g.sn
    omega = 1.3
    from oracle.greens import truncated_green_hat

    for name, d in (("xy", (1, -2, 2)), ("dx", (0, 1, -2))):
        kd = discrete.kernel_direct(name, g, omega)
        acc = 0j
        half = (sn - 1) // 2
        for mz in range(-half, half + 1):
            for my in range(-half, half + 1):
                for mx in range(-half, half + 1):
                    kz, ky, kx = (2 * np.pi * m / (3 * g.D) for m in (mz, my, mx))
                    kap = math.sqrt(kx * kx + ky * ky + kz * kz)
                    G = truncated_green_hat(np.array([kap]), omega, g.L)[0]
                    S = -kx * ky if name == "xy" else 1j * kx
                    acc += S * G * np.exp(2j * np.pi * (mz * d[0] + my * d[1] + mx * d[2]) / sn)
        acc /= sn ** 3
        got = kd[d[0] + 2, d[1] + 2, d[2] + 2]
        assert abs(got - acc) <= 1e-14 * max(1.0, abs(acc)), name


@pytest.mark.parametrize("name", ["1", "dx", "xx", "xz", "yz"])
def test_fft_convolution_equals_toeplitz(name):
    g = discrete.Grid(8)
    kt = discrete.KernelTransforms(g, 2.5)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((8, 8, 8)) + 1j * rng.standard_normal((8, 8, 8))
    y1 = kt.convolve(name, x)
    y2 = discrete.convolve_direct(discrete.kernel_direct(name, g, 2.5), x)
    assert np.linalg.norm(y1 - y2) <= 1e-14 * np.linalg.norm(y2) * 10


@pytest.mark.parametrize("n", [8, 5])
def test_kernel_parity_and_reality(n):
    g = discrete.Grid(n)
    n = g.n
    idx = (-np.arange(2 * n)) % (2 * n)
    for omega in (0.0, 2.0):
        for name in ("xx", "xy", "dz", "1"):
            e = discrete.kernel_fft(name, g, omega)
            flipped = e[np.ix_(idx, idx, idx)]
            odd = name in ("dx", "dy", "dz")
            assert np.max(np.abs(flipped - (-e if odd else e))) <= 1e-15 * np.max(np.abs(e)) * 10
            if omega == 0.0 and not odd:
                assert np.max(np.abs(e.imag)) <= 1e-15 * np.max(np.abs(e)) * 10


@pytest.mark.parametrize("n,tol", [(32, 2e-11), (48, 5e-15)])
def test_newton_potential_of_gaussian(n, tol):
    g = discrete.Grid(n)
    kt = discrete.KernelTransforms(g, 0.0)
    rho, r = gaussian(g)
    u = kt.convolve("1", rho + 0j)
    exact = sp.erf(np.sqrt(ALPHA) * r) / (4 * np.pi * r)
    assert np.max(np.abs(u - exact)) <= tol * np.max(exact)
    assert np.max(np.abs(u.imag)) <= 1e-15 * np.max(exact) * 10


def helmholtz_radial_potential(r_values, omega):
    """V_w rho(r) for the Gaussian by the l = 0 addition theorem, 1D adaptive quadrature."""
    rho = lambda s: (ALPHA / np.pi) ** 1.5 * np.exp(-ALPHA * s * s)
    out = []
    R = 1.5
    for r in r_values:
        inner_re = integrate.quad(lambda s: rho(s) * s * math.sin(omega * s), 0, r, epsabs=0, epsrel=1e-13, limit=200)[0]
        outer_re = integrate.quad(lambda s: rho(s) * s * math.cos(omega * s), r, R, epsabs=0, epsrel=1e-13, limit=200)[0]
        outer_im = integrate.quad(lambda s: rho(s) * s * math.sin(omega * s), r, R, epsabs=0, epsrel=1e-13, limit=200)[0]
        val = np.exp(1j * omega * r) / (omega * r) * inner_re + math.sin(omega * r) / (omega * r) * (outer_re + 1j * outer_im)
        out.append(val)
    return np.array(out)


def test_helmholtz_potential_of_gaussian():
    n, omega = 48, 4 * math.pi
    g = discrete.Grid(n)
    kt = discrete.KernelTransforms(g, omega)
    rho, r = gaussian(g)
    u = kt.convolve("1", rho + 0j)
    rng = np.random.default_rng(0)
    pts = rng.integers(0, n, size=(60, 3))
    rv = np.sqrt(sum(g.nodes()[pts[:, a]] ** 2 for a in range(3)))
    ref = helmholtz_radial_potential(rv, omega)
    got = u[pts[:, 0], pts[:, 1], pts[:, 2]]
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_laplacian_of_newton_potential():
    """Delta V_0 rho = -rho: the three diagonal -k_a^2 kernels summed act as -identity on rho."""
    g = discrete.Grid(48)
    kt = discrete.KernelTransforms(g, 0.0)
    rho, _ = gaussian(g)
    lap = sum(kt.convolve(nm, rho + 0j) for nm in ("xx", "yy", "zz"))
    assert np.max(np.abs(lap + rho)) <= 1e-12 * np.max(rho)


@pytest.mark.parametrize("omega", [0.0, 4 * math.pi])
def test_lemma2_gradient_and_curl(omega):
    """Lemma 2: 2 T grad psi = -grad psi; 2 T curl P = curl P (the curl part holds for every w)."""
    g = discrete.Grid(48)
    kt = discrete.KernelTransforms(g, omega)
    Z, Y, X = g.coords()
    psi = np.exp(-ALPHA * (X * X + Y * Y + Z * Z))
    curl = np.stack([-2 * ALPHA * Y * psi, 2 * ALPHA * X * psi, 0 * psi]) + 0j  # curl(psi e_z)
    T = operators.T_op(kt, curl)
    assert np.max(np.abs(2 * T - curl)) <= 1e-13 * np.max(np.abs(curl))
    if omega == 0.0:
        grad = np.stack([-2 * ALPHA * X * psi, -2 * ALPHA * Y * psi, -2 * ALPHA * Z * psi]) + 0j
        T = operators.T_op(kt, grad)
        assert np.max(np.abs(2 * T + grad)) <= 1e-13 * np.max(np.abs(grad))


def test_planted_symbol_sign_error_is_caught():
    """A plausible slip -- a flipped sign on -k_a k_b -- breaks the Lemma 2 pin by O(1)."""
    g = discrete.Grid(32)
    kt = discrete.KernelTransforms(g, 0.0)
    Z, Y, X = g.coords()
    psi = np.exp(-ALPHA * (X * X + Y * Y + Z * Z))
    grad = np.stack([-2 * ALPHA * X * psi, -2 * ALPHA * Y * psi, -2 * ALPHA * Z * psi]) + 0j
    for nm in ("xx", "yy", "zz", "xy", "xz", "yz"):
        kt._hat[nm] = -kt.hat(nm)  # planted mistake, in the oracle, on the CPU
    T = operators.T_op(kt, grad)
    assert np.max(np.abs(2 * T + grad)) > 0.5 * np.max(np.abs(grad))
