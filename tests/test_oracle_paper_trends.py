"""The oracle reproduces the qualitative findings of Sec. 5.2 (no GPU).

* The number of Bi-CGStab matvecs is about constant as the mesh is refined
  (the behaviour of a second-kind equation that Sec. 5.2 points out).
* Higher contrast needs more matvecs: eps234 (eigenvalues up to 1 + 3W) above
  eps222 (1 + W), as in Tables 2 and 3 (22 vs 37 matvecs at n = 70).
* More matvecs at higher frequency, and more at higher contrast for a fixed
  frequency (Fig. 2: Bi-CGStab iterations against w for the four media).
Both for the Helmholtz and the reduced Maxwell equations, one wavelength across
[0,1]^3 unless stated, E_in = (0, 0, exp(i w x)), tolerance 1e-12.
"""
import numpy as np
import pytest

import vie_inputs as vi
from oracle import operators, solvers


def matvecs(kind, medium, n):
    eps = vi.paper_medium(medium, n, 0.0, 1.0)
    op = operators.OracleProblem(kind, n, 0.0, 1.0, 2 * np.pi, eps)
    b = op.rhs(np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0]) if kind == "maxwell" else None)
    x, info = solvers.bicgstab(op.apply, b, tol=1e-12)
    assert info["converged"]
    return info["applies"]


@pytest.mark.parametrize("kind", ["helmholtz", "maxwell"])
def test_matvecs_mesh_independent_and_growing_with_contrast(kind):
    low = [matvecs(kind, "eps222", n) for n in (12, 18, 24)]
    high = [matvecs(kind, "eps234", n) for n in (12, 18, 24)]
    for counts in (low, high):
        assert max(counts) <= 1.1 * min(counts), counts
    assert min(high) > 1.4 * max(low), (low, high)


def matvecs_at(kind, medium, n, size):
    eps = vi.paper_medium(medium, n, 0.0, 1.0)
    op = operators.OracleProblem(kind, n, 0.0, 1.0, 2 * np.pi * size, eps)
    b = op.rhs(np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0]) if kind == "maxwell" else None)
    x, info = solvers.bicgstab(op.apply, b, tol=1e-12)
    assert info["converged"]
    return info["applies"]


@pytest.mark.parametrize("kind", ["helmholtz", "maxwell"])
def test_matvecs_grow_with_frequency_and_contrast(kind):
    """Fig. 2's trends: at a fixed medium the Bi-CGStab matvec count grows with
    w (half, one and two wavelengths across the box), and at a fixed w the
    locally isotropic high-contrast eps444 (eigenvalues up to 1 + 4W) needs more
    than eps222 (1 + W).  On a 16-grid the counts are 19/21/30 and 33/41/125
    (Helmholtz), 19/22/38 and 35/45/213 (reduced Maxwell)."""
    sizes = (0.5, 1.0, 2.0)
    low = [matvecs_at(kind, "eps222", 16, s) for s in sizes]
    high = [matvecs_at(kind, "eps444", 16, s) for s in sizes]
    for counts in (low, high):
        assert all(b > a for a, b in zip(counts, counts[1:])), counts
    assert all(h > 1.4 * lo for lo, h in zip(low, high)), (low, high)
    assert high[-1] > 2.5 * high[0], high  # the growth is strongest at high contrast
