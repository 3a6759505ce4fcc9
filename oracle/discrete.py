"""Discrete truncated-kernel convolutions on the uniform grid (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper discretises the volume potentials on a uniform n^3 grid and applies
them with the FFT after (a) truncating the Green's function, (b) transforming
it and (c) cutting the transform off at the grid's Nyquist frequency (Sec. 5).
The paper gives no further detail; the readings fixed here are:

* Grid: box [lo,hi]^3, D = hi - lo, h = D/n, cell-centred nodes.
* Truncation radius L = sqrt(3) D (the box diagonal, so every pair of nodes
  interacts through the untruncated kernel).
* Oversampling s = 3 (s D >= D + L needs s >= 1 + sqrt 3): the truncated
  kernel is expanded in a Fourier series of period sD, whose periodic images
  cannot reach the box, and the series is cut at |m_a| <= sn/2 (the grid
  Nyquist frequency pi/h).  For odd n (odd sn) the cut set is the symmetric
  |m_a| <= (sn-1)/2, which has no Nyquist entry.
* For a Fourier symbol S(k) in {1, i k_a, -k_a k_b} the discrete kernel on
  node offsets d in [-(n-1), n-1]^3 is

      K^S_d = (sD)^-3 sum_{m in [-sn/2, sn/2)^3} S~(k_m) G^_L(|k_m|) exp(i k_m . d h),
      k_m = 2 pi m / (sD),

  and (V_S x)_i = h^3 sum_j K^S_{i-j} x_j.  Nyquist rule: on an axis where
  m_a = -sn/2 the symbol is replaced by the mean of its values at
  k_a = -pi/h and +pi/h (odd factors k_a vanish there, k_a^2 is kept).

Because h / (sD) = 1/(sn), the weighted kernel kw_d = h^3 K^S_d is exactly the
normalised inverse DFT of size sn of the samples S~ G^, evaluated at d.

Two routes evaluate the same numbers:
* ``kernel_direct`` / ``convolve_direct``: the sums above written out
  (separable exponentials, Toeplitz matrix) -- the brute-force definition.
* ``kernel_fft`` / ``KernelTransforms.convolve``: the sums by library FFTs;
  the convolution by embedding kw cyclically in a (2n)^3 grid (index d mod 2n,
  index n left zero), which is an exact linear convolution for i, j < n.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass

import numpy as np
import scipy.fft as sfft

from .greens import truncated_green_hat

OVERSAMPLE = 3
WORKERS = os.cpu_count() or 1

AXES = {"x": 2, "y": 1, "z": 0}  # grid arrays are [z, y, x]
SYMBOLS = ("1", "dx", "dy", "dz", "xx", "yy", "zz", "xy", "xz", "yz")


@dataclass(frozen=True)
class Grid:
    """Uniform cell-centred grid on [lo, hi]^3 (Sec. 5: 'uniform n x n x n mesh')."""

    n: int
    lo: float = -1.0
    hi: float = 1.0

    @property
    def D(self) -> float:
        return self.hi - self.lo

    @property
    def h(self) -> float:
        return self.D / self.n

    @property
    def L(self) -> float:
        """Truncation radius: the box diagonal sqrt(3) D."""
        return math.sqrt(3.0) * self.D

    @property
    def sn(self) -> int:
        return OVERSAMPLE * self.n

    def nodes(self) -> np.ndarray:
        return self.lo + (np.arange(self.n) + 0.5) * self.h

    def coords(self):
        t = self.nodes()
        return t[:, None, None], t[None, :, None], t[None, None, :]


def _axis_wavenumbers(grid: Grid):
    """k along one axis in FFT order for the cutoff set of m; also k with the Nyquist entry zeroed.

    Even sn: m in [-sn/2, sn/2), and m = -sn/2 is the Nyquist entry.  Odd sn (odd n):
    m in [-(sn-1)/2, (sn-1)/2], symmetric, with no Nyquist entry to treat."""
    sn = grid.sn
    m = np.fft.fftfreq(sn, d=1.0 / sn)  # even sn: 0..sn/2-1, -sn/2..-1; odd sn: 0..(sn-1)/2, -(sn-1)/2..-1
    k = 2.0 * np.pi * m / (OVERSAMPLE * grid.D)
    k_odd = k.copy()
    if sn % 2 == 0:
        k_odd[sn // 2] = 0.0  # mean of S at k_a = -pi/h and +pi/h for odd factors
    return k, k_odd


def symbol_samples(name: str, grid: Grid):
    """S~(k_m) on the (sn)^3 grid, broadcastable, with the Nyquist rule applied."""
    k, k_odd = _axis_wavenumbers(grid)
    sn = grid.sn
    shape = {0: (sn, 1, 1), 1: (1, sn, 1), 2: (1, 1, sn)}

    def kk(axis_name, odd):
        ax = AXES[axis_name]
        return (k_odd if odd else k).reshape(shape[ax])

    if name == "1":
        return np.ones((1, 1, 1))
    if name in ("dx", "dy", "dz"):
        return 1j * kk(name[1], True)
    a, b = name[0], name[1]
    if a == b:
        return -(kk(a, False) ** 2) + 0j
    return -(kk(a, True) * kk(b, True)) + 0j


def green_samples(grid: Grid, omega: float) -> np.ndarray:
    """G^_L(|k_m|) on the full (sn)^3 grid (FFT order)."""
    k, _ = _axis_wavenumbers(grid)
    kappa = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    return truncated_green_hat(kappa, omega, grid.L)


def _offset_indices(grid: Grid):
    """(source index in the sn grid, destination index in the 2n grid) for d = 0..n-1, -(n-1)..-1."""
    n, sn = grid.n, grid.sn
    d = np.concatenate([np.arange(n), np.arange(-(n - 1), 0)])
    return d % sn, d % (2 * n), d


def kernel_fft(name: str, grid: Grid, omega: float, ghat: np.ndarray | None = None) -> np.ndarray:
    """Weighted kernel kw = h^3 K^S on the (2n)^3 embedding grid, via a size-sn inverse FFT."""
    if ghat is None:
        ghat = green_samples(grid, omega)
    F = symbol_samples(name, grid) * ghat
    kw_full = sfft.ifftn(F, workers=WORKERS)
    src, dst, _ = _offset_indices(grid)
    e = np.zeros((2 * grid.n,) * 3, np.complex128)
    e[np.ix_(dst, dst, dst)] = kw_full[np.ix_(src, src, src)]
    return e


def kernel_direct(name: str, grid: Grid, omega: float) -> np.ndarray:
    """Same kernel from the Fourier sum written out (no FFT); offsets d in [-(n-1), n-1]^3.

    Returned array is indexed [dz + n - 1, dy + n - 1, dx + n - 1].
    """
    sn = grid.sn
    m = np.fft.fftfreq(sn, d=1.0 / sn)
    d = np.arange(-(grid.n - 1), grid.n)
    E = np.exp(2j * np.pi * np.outer(d, m) / sn)  # [d, m]
    F = np.broadcast_to(symbol_samples(name, grid) * green_samples(grid, omega), (sn,) * 3)
    t = np.einsum("cq,abq->abc", E, F)  # x axis
    t = np.einsum("bp,apc->abc", E, t)  # y axis
    t = np.einsum("am,mbc->abc", E, t)  # z axis
    return t / float(sn) ** 3


def convolve_direct(kd: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y_i = sum_j kw_{i-j} x_j over the n^3 grid by an explicit Toeplitz matrix (small n only)."""
    n = x.shape[-1]
    idx = np.arange(n)
    I = np.stack(np.meshgrid(idx, idx, idx, indexing="ij"), -1).reshape(-1, 3)
    diff = I[:, None, :] - I[None, :, :] + (n - 1)
    T = kd[diff[..., 0], diff[..., 1], diff[..., 2]]
    return (T @ x.reshape(-1)).reshape(n, n, n)


class KernelTransforms:
    """DFT_{2n} of the embedded weighted kernels, computed on demand and cached."""

    def __init__(self, grid: Grid, omega: float):
        self.grid = grid
        self.omega = omega
        self._ghat = None
        self._hat: dict[str, np.ndarray] = {}

    def ghat(self):
        if self._ghat is None:
            self._ghat = green_samples(self.grid, self.omega)
        return self._ghat

    def embedded(self, name: str) -> np.ndarray:
        return kernel_fft(name, self.grid, self.omega, self.ghat())

    def hat(self, name: str) -> np.ndarray:
        if name not in self._hat:
            self._hat[name] = sfft.fftn(self.embedded(name), workers=WORKERS)
        return self._hat[name]

    def forward(self, x: np.ndarray) -> np.ndarray:
        """DFT_{2n} of x (n^3) zero-padded to (2n)^3."""
        n = self.grid.n
        p = np.zeros((2 * n,) * 3, np.complex128)
        p[:n, :n, :n] = x
        return sfft.fftn(p, workers=WORKERS)

    def backward(self, X: np.ndarray) -> np.ndarray:
        n = self.grid.n
        return sfft.ifftn(X, workers=WORKERS)[:n, :n, :n]

    def convolve(self, name: str, x: np.ndarray) -> np.ndarray:
        """(V_S x) on the n^3 grid."""
        return self.backward(self.hat(name) * self.forward(x))


def pair_name(a: int, b: int) -> str:
    """Symbol name for -k_a k_b with a, b in {0,1,2} = {x,y,z}."""
    s = "xyz"
    a, b = sorted((a, b))
    return s[a] + s[b]
