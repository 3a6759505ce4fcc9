"""Writes tests/golden/selfconv_oracle.json: self-convergence errors of the oracle.

The paper's Tables 2-5 report, beside the matvec counts, the L2 and L-infinity
errors E_2 and E_inf of the solution on the paper's media (Sec. 5.2, box
[0,1]^3, incident field E_in = (0, 0, exp(i w x))), which fall off
superalgebraically as the grid is refined (Sec. 5).  The tables do not say what
the errors are measured against.  Reading used here: the relative difference,
over all components of J, between the solution on an n-grid and the solution on
a grid r times finer (r odd, so that the cell-centred nodes nest), taken on the
n-grid's nodes:

    E_2   = ||J_n - J_rn|_nodes||_2 / ||J_rn|_nodes||_2
    E_inf = max |J_n - J_rn|_nodes| / max |J_rn|_nodes|

Every value here comes from the FP64 oracle (GMRES to 1e-13); nothing is read
from the CUDA library.  Run from the repository root:

    python tests/golden/make_selfconv.py
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import vie_inputs as vi  # noqa: E402
from oracle import operators, solvers  # noqa: E402

# (equation, medium, size = w / (2 pi), reference grid, coarse grids)
CASES = [
    ("maxwell", "eps222", 1.0, 60, [12, 20]),
    ("helmholtz", "eps234", 1.0, 60, [12, 20]),
]
DIRECTION = [1.0, 0.0, 0.0]
POLARISATION = [0.0, 0.0, 1.0]


def oracle_solution(kind, medium, size, n):
    eps = vi.paper_medium(medium, n, 0.0, 1.0)
    op = operators.OracleProblem(kind, n, 0.0, 1.0, 2 * np.pi * size, eps)
    b = op.rhs(np.array(DIRECTION), np.array(POLARISATION) if kind == "maxwell" else None)
    J, info = solvers.gmres(op.apply, b, tol=1e-13, restart=80)
    assert info["converged"], (kind, medium, n)
    return J


def main():
    rows = []
    for kind, medium, size, nref, coarse in CASES:
        Jr = oracle_solution(kind, medium, size, nref)
        for n in coarse:
            s = vi.nested_nodes(n, nref)
            ref = Jr[:, s, s, s]
            J = oracle_solution(kind, medium, size, n)
            rows.append({
                "equation": kind,
                "medium": medium,
                "size_wavelengths": size,
                "n": n,
                "n_ref": nref,
                "E2": float(np.linalg.norm(J - ref) / np.linalg.norm(ref)),
                "Einf": float(np.abs(J - ref).max() / np.abs(ref).max()),
            })
            print(rows[-1], flush=True)
    doc = {
        "source": "FP64 oracle (oracle/), written by tests/golden/make_selfconv.py",
        "cites": "Sec. 5.2 media and incident field; E_2 / E_inf columns of Tables 2-5",
        "reading": "relative L2 / L-inf difference of J on the coarse grid's nodes against the solution "
                   "on a grid n_ref / n (odd) times finer; box [0,1]^3, d = (1,0,0), p = (0,0,1); "
                   "oracle GMRES to 1e-13",
        "direction": DIRECTION,
        "polarisation": POLARISATION,
        "rows": rows,
    }
    with open(os.path.join(HERE, "selfconv_oracle.json"), "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
