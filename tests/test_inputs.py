"""The seeded input generators (vie_inputs) follow their definitions (no GPU).

* SplitMix64 (Steele, Lea and Flood 2014): the published first outputs for seed 0.
* Random rotations are proper orthogonal; directions are unit vectors;
  polarisations are an orthonormal pair perpendicular to the direction.
* The paper's media (Sec. 5.2): W is the product bump; eps222 / eps444 are
  (1 + W) I and (1 + 3 W) I; eps234 is diag(1 + W, 1 + 2 W, 1 + 3 W); eps_dense
  is that tensor rotated by R_2(pi x) R_1(pi y), so it is symmetric with the same
  eigenvalues at every node.
"""
import numpy as np

import vie_inputs as vi


def test_splitmix64_published_outputs():
    r = vi.SplitMix64(0)
    assert r.next_u64() == 0xE220A8397B1DCDAF
    assert r.next_u64() == 0x6E789E6AA1B965F4
    u = vi.SplitMix64(7)
    vals = [u.uniform() for _ in range(1000)]
    assert 0.0 <= min(vals) and max(vals) < 1.0 and abs(np.mean(vals) - 0.5) < 0.05


def test_rotations_directions_and_polarisations():
    rng = vi.SplitMix64(11)
    for _ in range(20):
        R = vi.random_rotation(rng)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14) and abs(np.linalg.det(R) - 1.0) < 1e-14
        d = vi.sphere_direction(rng)
        assert abs(np.linalg.norm(d) - 1.0) < 1e-14
        p1, p2 = vi.polarisations(d, rng.uniform() * 2 * np.pi)
        B = np.stack([d, p1, p2])
        assert np.allclose(B @ B.T, np.eye(3), atol=1e-14)


def test_paper_media_follow_their_definitions():
    n = 10
    W = vi.bump_W(n)
    Z, Y, X = vi.grid_coords(n, 0.0, 1.0)
    f = lambda t: np.exp(-(((t - 0.5) / 0.25) ** 8))
    assert np.allclose(W, f(X) * f(Y) * f(Z), rtol=0, atol=1e-15)
    eye = vi.identity_field(n)
    assert np.allclose(vi.paper_medium("eps222", n), eye * (1 + W), atol=1e-15)
    assert np.allclose(vi.paper_medium("eps444", n), eye * (1 + 3 * W), atol=1e-15)
    e234 = vi.paper_medium("eps234", n)
    for a in range(3):
        assert np.allclose(e234[a, a], 1 + (a + 1) * W, atol=1e-15)
    dense = vi.paper_medium("eps_dense", n)
    M = np.moveaxis(dense.real, (0, 1), (-2, -1)).reshape(-1, 3, 3)
    assert np.allclose(M, np.swapaxes(M, 1, 2), atol=1e-14) and np.max(np.abs(dense.imag)) == 0.0
    ev = np.sort(np.linalg.eigvalsh(M), axis=1)
    Wf = W.reshape(-1)
    assert np.allclose(ev, np.stack([1 + Wf, 1 + 2 * Wf, 1 + 3 * Wf], 1), atol=1e-13)
    # one node by hand: the rotation R_2(phi) R_1(theta) with phi = pi x, theta = pi y
    i = (3, 6, 2)  # (z, y, x)
    x, y = vi.grid_nodes(n, 0, 1)[i[2]], vi.grid_nodes(n, 0, 1)[i[1]]
    c1, s1, c2, s2 = np.cos(np.pi * y), np.sin(np.pi * y), np.cos(np.pi * x), np.sin(np.pi * x)
    R1 = np.array([[1, 0, 0], [0, c1, -s1], [0, s1, c1]])
    R2 = np.array([[c2, -s2, 0], [s2, c2, 0], [0, 0, 1]])
    w = W[i]
    D = np.diag([1 + w, 1 + 2 * w, 1 + 3 * w])
    assert np.allclose(dense[:, :, i[0], i[1], i[2]].real, R2 @ R1 @ D @ R1.T @ R2.T, atol=1e-14)


def test_oscillatory_medium_follows_its_definition():
    """Eq. (1stEx): (1 + W (1 + 0.1 sin(w x) sin(w y) sin(w z))) I; the device-side
    builder gives the same samples as the host one."""
    import torch

    n, w = 9, 40.0
    eps = vi.oscillatory_eps(n, w)
    i = (1, 4, 7)  # (z, y, x)
    t = vi.grid_nodes(n, 0.0, 1.0)
    z, y, x = t[i[0]], t[i[1]], t[i[2]]
    f = lambda s: np.exp(-(((s - 0.5) / 0.25) ** 8))
    v = 1.0 + f(x) * f(y) * f(z) * (1.0 + 0.1 * np.sin(w * x) * np.sin(w * y) * np.sin(w * z))
    assert np.allclose(eps[:, :, i[0], i[1], i[2]], v * np.eye(3), rtol=0, atol=1e-15)
    et = vi.oscillatory_eps_torch(n, "cpu", w).numpy()
    assert np.allclose(et, eps.reshape(9, -1), rtol=0, atol=1e-15)
    p = vi.oscillatory_problem(n, w)
    assert p.kind == "maxwell" and p.mu is None and (p.lo, p.hi, p.omega) == (0.0, 1.0, w)
    assert np.array_equal(p.directions[0], [1.0, 0.0, 0.0]) and np.array_equal(p.polarisations[0], [0.0, 0.0, 1.0])
