"""The oracle reproduces the qualitative findings of Sec. 5.2 (no GPU).

* The number of Bi-CGStab matvecs is about constant as the mesh is refined
  (the behaviour of a second-kind equation that Sec. 5.2 points out).
* Higher contrast needs more matvecs: eps234 (eigenvalues up to 1 + 3W) above
  eps222 (1 + W), as in Tables 2 and 3 (22 vs 37 matvecs at n = 70).
Both for the Helmholtz and the reduced Maxwell equations, one wavelength across
[0,1]^3, E_in = (0, 0, exp(i w x)), tolerance 1e-12.
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
