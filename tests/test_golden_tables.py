"""The transcribed Tables 2-5 of the paper (tests/golden/paper_tables.json) are self-consistent.

The fixture is used by ``bench.py --legs paper`` to set the matvec counts this
library's Bi-CGStab needs on the paper's media beside the printed ones.
"""
import json
import os

import numpy as np

import vie_inputs as vi

HERE = os.path.dirname(os.path.abspath(__file__))


def load():
    with open(os.path.join(HERE, "golden", "paper_tables.json")) as f:
        return json.load(f)


def test_fixture_shape_and_unknown_counts():
    doc = load()
    rows = doc["rows"]
    assert len(rows) == 52
    assert {r["medium"] for r in rows} == {"eps222", "eps234", "eps_dense", "eps444"}
    for r in rows:
        # N_tot = 3 n^3 to the three digits the tables print
        assert abs(r["N_tot"] - 3 * r["n"] ** 3) <= 0.006 * r["N_tot"]
        assert r["N_matvec"] > 0 and r["time_s"] > 0


def test_matvec_counts_mesh_independent_as_stated():
    """Sec. 5.2: the iteration count is about constant as the mesh is refined."""
    rows = load()["rows"]
    groups = {}
    for r in rows:
        groups.setdefault((r["medium"], r["size_wavelengths"]), []).append(r["N_matvec"])
    for key, counts in groups.items():
        assert max(counts) <= 1.2 * min(counts), key


def test_paper_media_generators():
    """eps222/444 isotropic with contrast 2/4; eps234 diagonal; eps_dense = R eps234 R^T (same eigenvalues)."""
    n = 12
    W = vi.bump_W(n)
    e222 = vi.paper_medium("eps222", n)
    e444 = vi.paper_medium("eps444", n)
    e234 = vi.paper_medium("eps234", n)
    ed = vi.paper_medium("eps_dense", n)
    assert np.allclose(e222[0, 0], 1 + W) and np.allclose(e444[2, 2], 1 + 3 * W)
    assert np.allclose(e234[1, 1], 1 + 2 * W) and np.allclose(e234[0, 1], 0)
    A = np.moveaxis(ed.real, (0, 1), (-2, -1)).reshape(-1, 3, 3)
    B = np.moveaxis(e234.real, (0, 1), (-2, -1)).reshape(-1, 3, 3)
    assert np.allclose(np.linalg.eigvalsh(A), np.linalg.eigvalsh(B), atol=1e-12)
    assert np.allclose(A, np.swapaxes(A, -1, -2))
    assert np.max(W) <= 1.0 and W[0, 0, 0] < 1e-15  # vanishes at the box edge
