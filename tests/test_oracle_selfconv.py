"""Self-convergence of the oracle on the paper's media (Sec. 5, Sec. 5.2).

Sec. 5 states that, for data resolved on the mesh, the truncated-kernel Fourier
method converges superalgebraically, and Tables 2-5 show the error falling by
orders of magnitude between n = 70, 120 and 180.  The oracle must show the same
behaviour: a mistake whose size depends on the grid (a wrong power of h, a
cutoff tied to the wrong index, a shifted node) makes solutions on nested grids
stop agreeing.  The stored values in tests/golden/selfconv_oracle.json (written
by tests/golden/make_selfconv.py from the oracle alone) are the targets of the
GPU test of the same study.
"""
import json
import os

import numpy as np
import pytest

import vie_inputs as vi
from oracle import operators, solvers

HERE = os.path.dirname(os.path.abspath(__file__))


def test_nested_nodes_pick_coincident_nodes():
    for n, r in [(6, 7), (12, 5), (20, 3), (70, 3), (9, 1)]:
        s = vi.nested_nodes(n, r * n)
        assert np.allclose(vi.grid_nodes(r * n, 0.0, 1.0)[s], vi.grid_nodes(n, 0.0, 1.0), rtol=0, atol=1e-15)
        assert np.allclose(vi.grid_nodes(r * n, -1.0, 1.0)[s], vi.grid_nodes(n, -1.0, 1.0), rtol=0, atol=1e-15)
    for n, m in [(10, 20), (12, 30), (0, 10)]:
        with pytest.raises(ValueError):
            vi.nested_nodes(n, m)


def _solve(kind, medium, size, n):
    eps = vi.paper_medium(medium, n, 0.0, 1.0)
    op = operators.OracleProblem(kind, n, 0.0, 1.0, 2 * np.pi * size, eps)
    b = op.rhs(np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0]) if kind == "maxwell" else None)
    J, info = solvers.gmres(op.apply, b, tol=1e-13, restart=80)
    assert info["converged"]
    return J


def test_oracle_self_converges_on_eps222():
    """Reduced Maxwell on eps222, one wavelength across the box: the error of the
    6- and 14-grid solutions against the 42-grid one drops by more than an order
    of magnitude (smooth bump medium, Sec. 5.2)."""
    Jr = _solve("maxwell", "eps222", 1.0, 42)
    errs = []
    for n in (6, 14):
        s = vi.nested_nodes(n, 42)
        ref = Jr[:, s, s, s]
        errs.append(np.linalg.norm(_solve("maxwell", "eps222", 1.0, n) - ref) / np.linalg.norm(ref))
    assert errs[1] < errs[0] / 10
    assert errs[1] < 1e-2


def test_stored_study_decreases_with_n():
    with open(os.path.join(HERE, "golden", "selfconv_oracle.json")) as f:
        rows = json.load(f)["rows"]
    groups = {}
    for r in rows:
        groups.setdefault((r["equation"], r["medium"], r["size_wavelengths"], r["n_ref"]), []).append(r)
    assert len(groups) == 2
    for key, rs in groups.items():
        rs.sort(key=lambda r: r["n"])
        for a, b in zip(rs, rs[1:]):
            assert b["E2"] < a["E2"] / 4 and b["Einf"] < a["Einf"] / 4, key
