"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module only draws random numbers and samples the media and incident
directions that define a scattering problem.  It holds none of the method's
arithmetic (no H tensors, no kernels, no operators, no right-hand sides):
those are computed separately, and independently, by the oracle and by the
CUDA library.

Conventions
-----------
* Box ``[lo, hi]^3``, ``D = hi - lo``, ``h = D / n``.  Grid nodes are cell
  centred, ``x_i = lo + (i + 1/2) h`` (the paper only says "uniform n x n x n
  mesh", Sec. 5; cell centring is the reading used throughout).
* Grid arrays are indexed ``[z, y, x]`` with ``x`` fastest.
* A 3x3 medium tensor field is a complex128 array of shape ``(3, 3, n, n, n)``
  (row index, column index, z, y, x); flattened it is the ``[9][n][n][n]``
  layout the C ABI takes.
* Random numbers come from SplitMix64 (Steele, Lea, Flood 2014); a uniform
  double is ``(x >> 11) * 2^-53``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (Steele, Lea and Flood, OOPSLA 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_range(self, a: float, b: float) -> float:
        return a + (b - a) * self.uniform()

    def normals(self, count: int) -> np.ndarray:
        """Box-Muller standard normals (used only for random test vectors)."""
        out = np.empty(count)
        for i in range(0, count, 2):
            u1 = max(self.uniform(), 1e-300)
            u2 = self.uniform()
            r = math.sqrt(-2.0 * math.log(u1))
            out[i] = r * math.cos(2 * math.pi * u2)
            if i + 1 < count:
                out[i + 1] = r * math.sin(2 * math.pi * u2)
        return out


def random_rotation(rng: SplitMix64) -> np.ndarray:
    """Uniform random rotation from a unit quaternion (Shoemake, Graphics Gems III)."""
    u1, u2, u3 = rng.uniform(), rng.uniform(), rng.uniform()
    a = math.sqrt(1.0 - u1)
    b = math.sqrt(u1)
    qx, qy = a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2)
    qz, qw = b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)
    return np.array([
        [1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)],
        [2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)],
        [2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)],
    ])


def sphere_direction(rng: SplitMix64) -> np.ndarray:
    """Uniform unit vector: z = 2u - 1, azimuth = 2 pi u."""
    z = 2.0 * rng.uniform() - 1.0
    phi = 2.0 * math.pi * rng.uniform()
    s = math.sqrt(max(0.0, 1.0 - z * z))
    return np.array([s * math.cos(phi), s * math.sin(phi), z])


def polarisations(d: np.ndarray, angle: float) -> tuple[np.ndarray, np.ndarray]:
    """Two orthonormal unit vectors perpendicular to ``d``, rotated by ``angle``."""
    helper = np.array([1.0, 0.0, 0.0]) if abs(d[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = helper - d * (helper @ d)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    c, s = math.cos(angle), math.sin(angle)
    return c * e1 + s * e2, -s * e1 + c * e2


def grid_nodes(n: int, lo: float, hi: float) -> np.ndarray:
    """Cell-centred node coordinates along one axis."""
    h = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * h


def grid_coords(n: int, lo: float, hi: float):
    """Broadcastable (Z, Y, X) coordinate arrays of shape (n,1,1), (1,n,1), (1,1,n)."""
    t = grid_nodes(n, lo, hi)
    return t[:, None, None], t[None, :, None], t[None, None, :]


def nested_nodes(n_coarse: int, n_fine: int) -> slice:
    """Per-axis slice of an n_fine grid that picks the nodes of the n_coarse grid.

    Cell-centred grids nest only for an odd ratio r = n_fine / n_coarse: coarse
    node i, at lo + (i + 1/2) D / n_coarse, is fine node r i + (r - 1) / 2.  Used
    to compare solutions on two grids (a self-convergence study) without
    interpolation."""
    r = n_fine // n_coarse if n_coarse >= 1 else 0
    if r < 1 or r * n_coarse != n_fine or r % 2 == 0:
        raise ValueError(f"grids {n_coarse} and {n_fine} do not nest (need an odd integer ratio)")
    return slice((r - 1) // 2, None, r)


def _tensor_field(weight: np.ndarray, mat: np.ndarray) -> np.ndarray:
    """weight (n,n,n) real times a constant 3x3 matrix -> (3,3,n,n,n)."""
    return mat.astype(np.complex128)[:, :, None, None, None] * weight[None, None]


def identity_field(n: int) -> np.ndarray:
    eye = np.zeros((3, 3, n, n, n), np.complex128)
    for a in range(3):
        eye[a, a] = 1.0
    return eye


# --------------------------------------------------------------------------
# Problem descriptions
# --------------------------------------------------------------------------


@dataclass
class Problem:
    """A synthetic scattering problem: medium samples plus incident-wave data."""

    kind: str  # "laplace" | "helmholtz" | "maxwell"
    n: int
    lo: float
    hi: float
    omega: float
    eps: np.ndarray  # (3,3,n,n,n) complex128
    mu: np.ndarray | None  # (3,3,n,n,n) complex128 or None (identity)
    directions: np.ndarray  # (nrhs, 3) unit propagation directions (Laplace: field direction)
    polarisations: np.ndarray  # (nrhs, 3) unit polarisations (Maxwell) / zeros
    meta: dict = field(default_factory=dict)

    @property
    def nrhs(self) -> int:
        return self.directions.shape[0]


def anisotropic_bump(n, lo, hi, amp, width2, rng, eig=(1.0, 2.0, 3.0), eig_imag=None):
    """I + amp * exp(-|x|^2 / width2) * R diag(eig) R^T with a seeded rotation R."""
    Z, Y, X = grid_coords(n, lo, hi)
    g = np.exp(-(X * X + Y * Y + Z * Z) / width2)
    R = random_rotation(rng)
    lam = np.array(eig, dtype=np.complex128)
    if eig_imag is not None:
        lam = lam + 1j * np.asarray(eig_imag)
    S = R @ np.diag(lam) @ R.T
    return identity_field(n) + amp * _tensor_field(g, S)


def laplace_bump_problem(n=32, seed=0, lo=-1.0, hi=1.0, E0=(0.0, 0.0, 1.0)) -> Problem:
    """Electrostatic workload: eps = I + 0.5 exp(-|x|^2/0.1) R diag(1,2,3) R^T, uniform field E0."""
    rng = SplitMix64(seed)
    eps = anisotropic_bump(n, lo, hi, 0.5, 0.1, rng).real.astype(np.complex128)
    return Problem("laplace", n, lo, hi, 0.0, eps, None,
                   np.array([E0], dtype=np.float64), np.zeros((1, 3)),
                   meta={"workload": f"laplace_bump_{n}", "seed": seed})


def helmholtz_multibump_medium(n, seed, lo=-1.0, hi=1.0, nbumps=4, lossless=False):
    """eps = I + sum_j a_j exp(-|x-c_j|^2/sigma_j^2) Q_j diag(lam_j) Q_j^T (complex symmetric).

    a_j ~ U[0.5,1]; c_j uniform in the ball |c|<0.5; sigma_j ~ U[0.15,0.3];
    Re lam ~ U[0.5,2], Im lam ~ U[0,0.05]; Q_j a seeded rotation.
    """
    rng = SplitMix64(seed)
    Z, Y, X = grid_coords(n, lo, hi)
    eps = identity_field(n)
    for _ in range(nbumps):
        a = rng.uniform_range(0.5, 1.0)
        while True:
            c = np.array([rng.uniform_range(-0.5, 0.5) for _ in range(3)])
            if c @ c < 0.25:
                break
        sigma = rng.uniform_range(0.15, 0.3)
        Q = random_rotation(rng)
        lam = np.array([rng.uniform_range(0.5, 2.0) + 1j * rng.uniform_range(0.0, 0.05) for _ in range(3)])
        if lossless:
            lam = lam.real.astype(np.complex128)
        S = Q @ np.diag(lam) @ Q.T
        g = np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / sigma ** 2)
        eps = eps + a * _tensor_field(g, S)
    return eps, rng


def helmholtz_problem(n=128, seed=0, wavelengths=4.0, lo=-1.0, hi=1.0, nrhs=1, lossless=False) -> Problem:
    """Acoustic workload: multi-bump complex-symmetric medium, plane wave along seeded d."""
    eps, rng = helmholtz_multibump_medium(n, seed, lo, hi, lossless=lossless)
    omega = 2.0 * math.pi * wavelengths / (hi - lo)
    dirs = np.array([sphere_direction(rng) for _ in range(nrhs)])
    return Problem("helmholtz", n, lo, hi, omega, eps, None, dirs, np.zeros((nrhs, 3)),
                   meta={"workload": f"helmholtz_multibump_{n}", "seed": seed,
                         "wavelengths": wavelengths})


def maxwell_problem(n=256, seed=0, wavelengths=10.0, lo=-1.0, hi=1.0, ndirs=1, npol=1,
                    with_mu=True, eta_max=0.05) -> Problem:
    """Electromagnetic workload: eps = I + 0.5 g S_eps, mu = I + 0.3 g S_mu.

    g = exp(-|x|^2/0.1); S = R diag(1+i eta1, 2+i eta2, 3+i eta3) R^T, eta ~ U[0, eta_max];
    eps is drawn first, then mu, then the incident directions and polarisation angles.
    """
    rng = SplitMix64(seed)
    eta_e = [rng.uniform_range(0.0, eta_max) for _ in range(3)]
    eps = anisotropic_bump(n, lo, hi, 0.5, 0.1, rng, eig_imag=eta_e)
    mu = None
    if with_mu:
        eta_m = [rng.uniform_range(0.0, eta_max) for _ in range(3)]
        mu = anisotropic_bump(n, lo, hi, 0.3, 0.1, rng, eig_imag=eta_m)
    omega = 2.0 * math.pi * wavelengths / (hi - lo)
    dirs, pols = [], []
    for _ in range(ndirs):
        d = sphere_direction(rng)
        angle = 2.0 * math.pi * rng.uniform()
        p1, p2 = polarisations(d, angle)
        for p in (p1, p2)[:npol]:
            dirs.append(d)
            pols.append(p)
    return Problem("maxwell", n, lo, hi, omega, eps, mu, np.array(dirs), np.array(pols),
                   meta={"workload": f"maxwell_bump_{n}", "seed": seed, "wavelengths": wavelengths})


# --------------------------------------------------------------------------
# The paper's own media (Sec. 5.2), on the unit box [0,1]^3
# --------------------------------------------------------------------------


def bump_W(n, lo=0.0, hi=1.0):
    """W(x,y,z) = prod_i exp(-((x_i - 0.5)/0.25)^8) (Sec. 5), zero to machine precision at the box edge."""
    Z, Y, X = grid_coords(n, lo, hi)
    f = lambda t: np.exp(-(((t - 0.5) / 0.25) ** 8))
    return f(X) * f(Y) * f(Z)


def paper_medium(name: str, n: int, lo=0.0, hi=1.0) -> np.ndarray:
    """eps222, eps444, eps234 or eps_dense of Sec. 5.2 sampled on the grid."""
    W = bump_W(n, lo, hi)
    eps = np.zeros((3, 3, n, n, n), np.complex128)
    if name == "eps222":
        for a in range(3):
            eps[a, a] = 1.0 + W
        return eps
    if name == "eps444":
        for a in range(3):
            eps[a, a] = 1.0 + 3.0 * W
        return eps
    diag = [1.0 + W, 1.0 + 2.0 * W, 1.0 + 3.0 * W]
    if name == "eps234":
        for a in range(3):
            eps[a, a] = diag[a]
        return eps
    if name == "eps_dense":
        Z, Y, X = grid_coords(n, lo, hi)
        phi = np.pi * X + 0 * Y + 0 * Z
        theta = np.pi * Y + 0 * X + 0 * Z
        c1, s1 = np.cos(theta), np.sin(theta)
        c2, s2 = np.cos(phi), np.sin(phi)
        one, zero = np.ones_like(W), np.zeros_like(W)
        R1 = np.array([[one, zero, zero], [zero, c1, -s1], [zero, s1, c1]])
        R2 = np.array([[c2, -s2, zero], [s2, c2, zero], [zero, zero, one]])
        R = np.einsum("ab...,bc...->ac...", R2, R1)
        Dm = np.array([[diag[0], zero, zero], [zero, diag[1], zero], [zero, zero, diag[2]]])
        eps = np.einsum("ab...,bc...,dc...->ad...", R, Dm, R)
        return eps.astype(np.complex128)
    raise ValueError(name)


def oscillatory_eps(n: int, omega: float = 408.0, lo=0.0, hi=1.0) -> np.ndarray:
    """(1 + W (1 + 0.1 sin(omega x) sin(omega y) sin(omega z))) I, the isotropic
    oscillatory medium of the first experiment of Sec. 5.2 (Eq. (1stEx))."""
    Z, Y, X = grid_coords(n, lo, hi)
    s = 1.0 + bump_W(n, lo, hi) * (1.0 + 0.1 * np.sin(omega * X) * np.sin(omega * Y) * np.sin(omega * Z))
    eps = np.zeros((3, 3, n, n, n), np.complex128)
    for a in range(3):
        eps[a, a] = s
    return eps


def oscillatory_problem(n: int, omega: float = 408.0) -> Problem:
    """Reduced Maxwell (mu = I) on [0,1]^3 with ``oscillatory_eps`` and the incident
    wave E^in = (0, 0, exp(i omega x)) of the first experiment of Sec. 5.2."""
    return Problem("maxwell", n, 0.0, 1.0, omega, oscillatory_eps(n, omega), None,
                   np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 0.0, 1.0]]),
                   meta={"workload": f"maxwell_oscillatory_{n}", "omega": omega})


def random_field(n: int, c: int, seed: int, nrhs: int = 1) -> np.ndarray:
    """Seeded complex Gaussian test vector of shape (nrhs, c, n, n, n) (numpy generator)."""
    g = np.random.default_rng(seed)
    shape = (nrhs, c, n, n, n)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def smooth_sphere_eps(n, eps_s, radius, delta, lo=-1.0, hi=1.0):
    """Isotropic eps = 1 + (eps_s - 1) * s(r), s a smooth step of width delta at r = radius."""
    import scipy.special as sp

    Z, Y, X = grid_coords(n, lo, hi)
    r = np.sqrt(X * X + Y * Y + Z * Z)
    s = 0.5 * sp.erfc((r - radius) / delta)
    eps = np.zeros((3, 3, n, n, n), np.complex128)
    for a in range(3):
        eps[a, a] = 1.0 + (eps_s - 1.0) * s
    return eps


# --------------------------------------------------------------------------
# Device-side generation (serving): the same formula as ``anisotropic_bump``,
# evaluated with torch on the device so that a request's medium never crosses
# the host link.  Still input generation only: no method arithmetic.
# --------------------------------------------------------------------------


def bump_medium_torch(n: int, seed: int, device, lo=-1.0, hi=1.0, amp=0.5, width2=0.1, eig=(1.0, 2.0, 3.0)):
    """[9][n^3] complex128 torch tensor of I + amp exp(-|x|^2/width2) R diag(eig) R^T (R from SplitMix64(seed))."""
    import torch

    rng = SplitMix64(seed)
    R = random_rotation(rng)
    S = R @ np.diag(np.asarray(eig, dtype=np.float64)) @ R.T
    t = torch.as_tensor(grid_nodes(n, lo, hi), dtype=torch.float64, device=device)
    r2 = t[:, None, None] ** 2 + t[None, :, None] ** 2 + t[None, None, :] ** 2
    g = torch.exp(-r2 / width2).reshape(-1)
    eps = torch.zeros((9, n * n * n), dtype=torch.complex128, device=device)
    for a in range(3):
        for b in range(3):
            eps[3 * a + b] = amp * float(S[a, b]) * g + (1.0 if a == b else 0.0)
    return eps


def oscillatory_eps_torch(n: int, device, omega: float = 408.0, lo=0.0, hi=1.0):
    """[9][n^3] complex128 torch tensor of ``oscillatory_eps`` built on the device
    (at n = 326 the host array would be 5 GB)."""
    import torch

    t = torch.as_tensor(grid_nodes(n, lo, hi), dtype=torch.float64, device=device)
    f = torch.exp(-(((t - 0.5) / 0.25) ** 8))
    sw = torch.sin(omega * t)
    W = (f[:, None, None] * f[None, :, None] * f[None, None, :]).reshape(-1)
    osc = (sw[:, None, None] * sw[None, :, None] * sw[None, None, :]).reshape(-1)
    s = 1.0 + W * (1.0 + 0.1 * osc)
    eps = torch.zeros((9, n * n * n), dtype=torch.complex128, device=device)
    for a in range(3):
        eps[4 * a] = s
    return eps


@dataclass
class ServeRequest:
    """One solve request of the serving mix."""

    rid: int
    arrival_s: float
    kind: str  # "helmholtz" | "maxwell"
    n: int
    wavelengths: float
    seed: int
    direction: np.ndarray
    polarisation: np.ndarray


def serving_mix(count: int, rate_per_s: float, seed: int = 0, sizes=(32, 48, 64, 96, 128, 192),
                wl_range=(1.0, 8.0), lo=-1.0, hi=1.0):
    """Poisson arrivals at ``rate_per_s``; n uniform over ``sizes``; wavelengths across
    the box uniform in ``wl_range``; kind Helmholtz / Maxwell (mu = I) 50/50; media from
    the anisotropic-bump generator with a per-request seed."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for i in range(count):
        u = max(rng.uniform(), 1e-300)
        t += -math.log(u) / rate_per_s
        n = sizes[min(len(sizes) - 1, int(rng.uniform() * len(sizes)))]
        wl = rng.uniform_range(*wl_range)
        kind = "helmholtz" if rng.uniform() < 0.5 else "maxwell"
        d = sphere_direction(rng)
        p, _ = polarisations(d, 2 * math.pi * rng.uniform())
        out.append(ServeRequest(i, t, kind, n, wl, 1000 + i, d, p))
    return out
