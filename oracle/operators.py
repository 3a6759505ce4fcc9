"""Operators I+B+K, right-hand sides and scattered fields (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Vectors are complex128 arrays of shape (c, n, n, n): component (x, y, z, and
for the coupled Maxwell system the M components after the J components),
then the grid [z, y, x].

Operators (the discrete V_S of ``discrete`` stand in for the volume potentials):
* W J := grad div V J, component a = sum_b V_{-k_a k_b} J_b.
* T J := J/2 + W J                                   (Eq. (Todef), Eq. (Vw)).
* Laplace  (Eq. (eq:intLap)):  J - 2 H_eps T_0 J           = 2 H_eps grad phi_in.
* Helmholtz (Eqs. (contractionK)-(eq:intH)): the derivation in the proof of the
  existence theorem of Sec. 3 multiplies by -2 (eps^-1 + I)^-1, which gives
      J - 2 H_{eps^-1} T_w J = 2 H_{eps^-1} grad phi_in.
  The printed Eq. (eq:intH) carries "+2H"; the sign here is the one the
  derivation produces (and the one Eqs. (eq:intLap) and (eq:intM) carry).
* Maxwell (Eq. (eq:intM)), unknowns J = J_V/(-i w), M = M_V/(-i w):
      J - 2 H_eps (T J + w^2 V J + i w curl V M) = 2 H_eps E_in
      M - 2 H_mu  (T M + w^2 V M - i w curl V J) = 2 H_mu  H_in
  With mu = I the second row gives M = 0 and the first is Eq.
  (contraction_Maxwell_reduced); that reduced 3-component system is what
  ``apply_maxwell(..., Hmu=None)`` computes.
Scattered fields: phi_sc = div V J (Sec. 2 existence proof, Eq. (eq:intH)
summary); E_sc, H_sc by Eq. (represent_Maxwell) / (represent_Maxwell_reduced).
Incident fields: Laplace grad phi_in = -E0 (reading: E = -grad phi); Helmholtz
phi_in = exp(i w d.x); Maxwell E_in = p exp(i w d.x), H_in = (d x p) exp(i w d.x)
(time dependence exp(-i w t), consistent with Eq. (Maxwell0)).
"""
from __future__ import annotations

import numpy as np

from .discrete import Grid, KernelTransforms, pair_name


def _eye_field(shape_tail):
    e = np.zeros((3, 3) + shape_tail, np.complex128)
    for a in range(3):
        e[a, a] = 1.0
    return e


def h_tensor(eps: np.ndarray) -> np.ndarray:
    """H_eps = (eps + I)^-1 (eps - I) at every node (Eq. (rhodef)); eps shape (3,3,n,n,n)."""
    I = _eye_field(eps.shape[2:])
    A = np.moveaxis(eps + I, (0, 1), (-2, -1))
    B = np.moveaxis(eps - I, (0, 1), (-2, -1))
    H = np.linalg.solve(A, B)
    return np.moveaxis(H, (-2, -1), (0, 1))


def inverse_field(eps: np.ndarray) -> np.ndarray:
    """eps^-1 at every node."""
    A = np.moveaxis(eps, (0, 1), (-2, -1))
    return np.moveaxis(np.linalg.inv(A), (-2, -1), (0, 1))


def tmul(H: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Pointwise 3x3 tensor times 3-vector field."""
    return np.einsum("ab...,b...->a...", H, x)


def grad_div_V(kt: KernelTransforms, x: np.ndarray) -> np.ndarray:
    """W x = grad div V x, component a = sum_b V_{-k_a k_b} x_b."""
    X = [kt.forward(x[b]) for b in range(3)]
    out = np.empty_like(x)
    for a in range(3):
        acc = sum(kt.hat(pair_name(a, b)) * X[b] for b in range(3))
        out[a] = kt.backward(acc)
    return out


def T_op(kt: KernelTransforms, x: np.ndarray) -> np.ndarray:
    """T x = x/2 + grad div V x (Eq. (Todef); Eq. (Vw) for w != 0)."""
    return 0.5 * x + grad_div_V(kt, x)


def V_op(kt: KernelTransforms, x: np.ndarray) -> np.ndarray:
    return np.stack([kt.convolve("1", x[a]) for a in range(x.shape[0])])


def curl_V(kt: KernelTransforms, x: np.ndarray) -> np.ndarray:
    """curl V x: (curl V x)_a = sum eps_abc d_b V x_c (symbol i k_b)."""
    X = [kt.forward(x[c]) for c in range(3)]
    D = {0: kt.hat("dx"), 1: kt.hat("dy"), 2: kt.hat("dz")}
    out = np.empty_like(x)
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        out[a] = kt.backward(D[b] * X[c] - D[c] * X[b])
    return out


def div_V(kt: KernelTransforms, x: np.ndarray) -> np.ndarray:
    """div V x = sum_a V_{i k_a} x_a (scalar field)."""
    names = ("dx", "dy", "dz")
    return kt.backward(sum(kt.hat(names[a]) * kt.forward(x[a]) for a in range(3)))


# ---------------------------------------------------------------- operators


def apply_laplace(kt: KernelTransforms, H: np.ndarray, J: np.ndarray) -> np.ndarray:
    """(I + B) J with B = -2 H_eps T_0 (Eq. (eq:intLap))."""
    return J - 2.0 * tmul(H, T_op(kt, J))


def apply_helmholtz(kt: KernelTransforms, Hinv: np.ndarray, J: np.ndarray) -> np.ndarray:
    """J - 2 H_{eps^-1} T_w J (Eq. (eq:intH) with the derived sign); Hinv = H_{eps^-1}."""
    return J - 2.0 * tmul(Hinv, T_op(kt, J))


def apply_maxwell(kt: KernelTransforms, He: np.ndarray, Hmu: np.ndarray | None, JM: np.ndarray) -> np.ndarray:
    """Eq. (eq:intM) on [J; M] (6 components), or Eq. (contraction_Maxwell_reduced) on J if Hmu is None."""
    w = kt.omega
    if Hmu is None:
        J = JM
        return J - 2.0 * tmul(He, T_op(kt, J) + w * w * V_op(kt, J))
    J, M = JM[:3], JM[3:]
    yJ = J - 2.0 * tmul(He, T_op(kt, J) + w * w * V_op(kt, J) + 1j * w * curl_V(kt, M))
    yM = M - 2.0 * tmul(Hmu, T_op(kt, M) + w * w * V_op(kt, M) - 1j * w * curl_V(kt, J))
    return np.concatenate([yJ, yM])


# ---------------------------------------------------------- incident fields


def plane_phase(grid: Grid, omega: float, d) -> np.ndarray:
    Z, Y, X = grid.coords()
    return np.exp(1j * omega * (d[0] * X + d[1] * Y + d[2] * Z))


def rhs_laplace(grid: Grid, H: np.ndarray, E0) -> np.ndarray:
    """2 H_eps grad phi_in with grad phi_in = -E0 uniform (Eq. (eq:intLap))."""
    n = grid.n
    g = np.stack([np.full((n, n, n), -float(E0[a]), np.complex128) for a in range(3)])
    return 2.0 * tmul(H, g)


def rhs_helmholtz(grid: Grid, Hinv: np.ndarray, omega: float, d) -> np.ndarray:
    """2 H_{eps^-1} grad phi_in, phi_in = exp(i w d.x) (Eq. (eq:intH))."""
    ph = plane_phase(grid, omega, d)
    g = np.stack([1j * omega * d[a] * ph for a in range(3)])
    return 2.0 * tmul(Hinv, g)


def rhs_maxwell(grid: Grid, He, Hmu, omega: float, d, p) -> np.ndarray:
    """[2 H_eps E_in; 2 H_mu H_in] (Eq. (eq:intM)); reduced (Hmu None): 2 H_eps E_in."""
    ph = plane_phase(grid, omega, d)
    E = np.stack([p[a] * ph for a in range(3)])
    b = 2.0 * tmul(He, E)
    if Hmu is None:
        return b
    q = np.cross(d, p)
    Hf = np.stack([q[a] * ph for a in range(3)])
    return np.concatenate([b, 2.0 * tmul(Hmu, Hf)])


# --------------------------------------------------------- scattered fields


def scattered_potential(kt: KernelTransforms, J: np.ndarray) -> np.ndarray:
    """phi_sc = div V J (Laplace: Sec. 2 existence proof; Helmholtz: summary after Eq. (eq:intH))."""
    return div_V(kt, J)


def scattered_em(kt: KernelTransforms, JM: np.ndarray, reduced: bool) -> np.ndarray:
    """[E_sc; H_sc] by Eq. (represent_Maxwell) (or (represent_Maxwell_reduced) when reduced)."""
    w = kt.omega
    if reduced:
        J = JM
        E = grad_div_V(kt, J) + w * w * V_op(kt, J)
        Hs = -1j * w * curl_V(kt, J)
        return np.concatenate([E, Hs])
    J, M = JM[:3], JM[3:]
    E = grad_div_V(kt, J) + w * w * V_op(kt, J) + 1j * w * curl_V(kt, M)
    Hs = grad_div_V(kt, M) + w * w * V_op(kt, M) - 1j * w * curl_V(kt, J)
    return np.concatenate([E, Hs])


# ------------------------------------------------------------ problem glue


class OracleProblem:
    """Bundles grid, H tensors and kernel transforms for one synthetic problem."""

    def __init__(self, kind: str, n: int, lo: float, hi: float, omega: float, eps, mu=None):
        self.kind = kind
        self.grid = Grid(n, lo, hi)
        self.omega = omega
        self.kt = KernelTransforms(self.grid, omega)
        self.eps = eps
        self.He = h_tensor(eps)
        self.Hinv = h_tensor(inverse_field(eps)) if kind == "helmholtz" else None
        self.Hmu = h_tensor(mu) if (kind == "maxwell" and mu is not None) else None

    @classmethod
    def from_problem(cls, p):
        return cls(p.kind, p.n, p.lo, p.hi, p.omega, p.eps, p.mu)

    @property
    def ncomp(self) -> int:
        return 6 if (self.kind == "maxwell" and self.Hmu is not None) else 3

    def apply(self, x: np.ndarray) -> np.ndarray:
        if self.kind == "laplace":
            return apply_laplace(self.kt, self.He, x)
        if self.kind == "helmholtz":
            return apply_helmholtz(self.kt, self.Hinv, x)
        return apply_maxwell(self.kt, self.He, self.Hmu, x)

    def rhs(self, d, p=None) -> np.ndarray:
        if self.kind == "laplace":
            return rhs_laplace(self.grid, self.He, d)
        if self.kind == "helmholtz":
            return rhs_helmholtz(self.grid, self.Hinv, self.omega, d)
        return rhs_maxwell(self.grid, self.He, self.Hmu, self.omega, d, p)

    def scattered(self, x: np.ndarray) -> np.ndarray:
        if self.kind in ("laplace", "helmholtz"):
            return scattered_potential(self.kt, x)[None]
        return scattered_em(self.kt, x, reduced=self.Hmu is None)
