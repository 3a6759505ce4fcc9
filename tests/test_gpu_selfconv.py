"""Self-convergence study on the paper's media through the C ABI (Sec. 5.2,
E_2 / E_inf columns of Tables 2-5).

The GPU solves the reduced Maxwell equation on eps222 and the Helmholtz equation
on eps234 (one wavelength across [0,1]^3, E_in = (0, 0, exp(i w x))) on 12-, 20-
and 60-grids; the errors of the coarse solutions against the 60-grid one, taken
on the nested nodes, must equal the oracle's (tests/golden/selfconv_oracle.json).
Both sides solve to at least 1e-12, so each error (about 1e-3 to 3e-2) is fixed to
better than 1e-8 of its value; the test allows 1e-6.
"""
import json
import os

import numpy as np
import pytest

import vie_inputs as vi
from gpu_common import to_dev, vie  # noqa: F401

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _gpu_solution(mod, kind, medium, size, n, d, pol):
    import torch

    eps = vi.paper_medium(medium, n, 0.0, 1.0)
    P = mod.Problem(kind, n, 0.0, 1.0, 2 * np.pi * size, to_dev(eps.reshape(9, -1)))
    try:
        b = torch.empty((3, n, n, n), dtype=torch.complex128, device="cuda:0")
        P.rhs(np.asarray(d), np.asarray(pol) if kind == "maxwell" else None, 1, b)
        J = torch.zeros_like(b)
        st, info = P.solve(b, J, tol=1e-12, restart=80, max_outer=40, mode=mod.VIE_SOLVE_FP64)
        assert info.rel_residual <= 1e-12
        return J.cpu().numpy()
    finally:
        P.close()


def test_self_convergence_matches_oracle(vie):
    with open(os.path.join(HERE, "golden", "selfconv_oracle.json")) as f:
        doc = json.load(f)
    refs = {}
    for row in doc["rows"]:
        key = (row["equation"], row["medium"], row["size_wavelengths"], row["n_ref"])
        if key not in refs:
            refs[key] = _gpu_solution(vie, *key, doc["direction"], doc["polarisation"])
        s = vi.nested_nodes(row["n"], row["n_ref"])
        ref = refs[key][:, s, s, s]
        J = _gpu_solution(vie, *key[:3], row["n"], doc["direction"], doc["polarisation"])
        e2 = np.linalg.norm(J - ref) / np.linalg.norm(ref)
        einf = np.abs(J - ref).max() / np.abs(ref).max()
        assert abs(e2 - row["E2"]) <= 1e-6 * row["E2"], (row, e2)
        assert abs(einf - row["Einf"]) <= 1e-6 * row["Einf"], (row, einf)
