"""GPU parity at grid sizes with a prime factor above 11.

For n = 13, 17, 26, 34 the set-up lines 3n (39, 51, 78, 102) do not factor
into the codelet radices 2, 3, 5, 7, 11: the set-up's kernel transforms run
Bluestein's chirp-z algorithm (a length-3n DFT as a circular convolution of
padded smooth length Q >= 6n - 1).  2n (26, 34, 52, 68) does not factor
either, so the apply runs on the padded convolution grid M = 2 nk (28, 36,
54, 70), nk the smallest smooth number >= n: a circular convolution of length
M >= 2n - 1 is the same zero-padded linear convolution on the n^3 nodes.  The
oracle transforms these lengths with numpy's FFT on the 2n grid.

Tolerances are those of the other parity tests: 1e-12 for FP64 and
double-word applies and the scattered field (a different grid length changes
only the rounding order), 2e-5 for FP32 applies, 1e-8 for solves stopped at a
relative residual of 1e-10.
"""
import numpy as np
import pytest

import vie_inputs as vi
from oracle import operators, solvers

from gpu_common import eps_dev, mu_dev, rel, to_dev, vie  # noqa: F401

pytestmark = pytest.mark.gpu

CASES = [
    ("laplace", 13, 0.0, False),
    ("helmholtz", 17, 2.0, False),
    ("helmholtz", 26, 3.0, False),
    ("maxwell", 13, 1.5, False),
    ("maxwell", 34, 2.0, True),
]
IDS = [f"{c[0]}-{c[1]}-mu{int(c[3])}" for c in CASES]


def _problem(kind, n, wl, with_mu, seed=0):
    if kind == "laplace":
        return vi.laplace_bump_problem(n=n, seed=seed)
    if kind == "helmholtz":
        return vi.helmholtz_problem(n=n, wavelengths=wl, seed=seed)
    return vi.maxwell_problem(n=n, wavelengths=wl, with_mu=with_mu, seed=seed)


_cache = {}


def _setup(vie, kind, n, wl, with_mu):
    key = (kind, n, wl, with_mu)
    if key not in _cache:
        p = _problem(kind, n, wl, with_mu)
        P = vie.Problem(kind, n, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
        _cache[key] = (p, P, operators.OracleProblem.from_problem(p))
    return _cache[key]


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_apply_fp64_bluestein(vie, case):
    import torch

    p, P, op = _setup(vie, *case)
    assert P.tune(vie.VIE_FP64) == -1  # generic kernels: no z-pass variant to pick
    x = vi.random_field(p.n, op.ncomp, 11)[0]
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    P.apply(xd, yd, vie.VIE_FP64)
    torch.cuda.synchronize()
    assert rel(yd.cpu().numpy(), op.apply(x)) <= 1e-12


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_apply_fp32_and_df64_bluestein(vie, case):
    import torch

    p, P, op = _setup(vie, *case)
    x = vi.random_field(p.n, op.ncomp, 12)[0]
    x32 = x.astype(np.complex64)
    y32 = torch.empty(x.shape, dtype=torch.complex64, device="cuda:0")
    P.apply(to_dev(x32), y32, vie.VIE_FP32)
    xd = to_dev(x)
    ydf = torch.empty_like(xd)
    P.apply(xd, ydf, vie.VIE_DF64)
    torch.cuda.synchronize()
    assert rel(y32.cpu().numpy(), op.apply(x32.astype(np.complex128))) <= 2e-5
    assert rel(ydf.cpu().numpy(), op.apply(x)) <= 1e-12


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_scattered_field_bluestein(vie, case):
    import torch

    p, P, op = _setup(vie, *case)
    x = vi.random_field(p.n, op.ncomp, 13)[0]
    cout = 1 if p.kind != "maxwell" else 6
    out = torch.empty((cout, p.n, p.n, p.n), dtype=torch.complex128, device="cuda:0")
    P.eval_scattered(to_dev(x), out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), op.scattered(x)) <= 1e-12


def test_batched_apply_equals_single_bluestein(vie):
    import torch

    p, P, op = _setup(vie, "helmholtz", 26, 3.0, False)
    x = vi.random_field(p.n, 3, 14, nrhs=2)
    xd = to_dev(x)
    yb = torch.empty_like(xd)
    P.apply(xd, yb, vie.VIE_FP64, nrhs=2)
    for r in range(2):
        ys = torch.empty_like(xd[r])
        P.apply(xd[r].contiguous(), ys, vie.VIE_FP64)
        torch.cuda.synchronize()
        assert torch.equal(ys, yb[r])


@pytest.mark.parametrize("case,mode", [(CASES[0], "mixed"), (CASES[2], "mixed"), (CASES[4], "mixed"),
                                       (CASES[3], "fp64")], ids=["laplace-13-mixed", "helmholtz-26-mixed",
                                                                 "maxwell-34-mu1-mixed", "maxwell-13-fp64"])
def test_solve_bluestein(vie, case, mode):
    import torch

    p, P, op = _setup(vie, *case)
    n = p.n
    b = torch.empty((P.ncomp, n, n, n), dtype=torch.complex128, device="cuda:0")
    pol = p.polarisations[0] if p.kind == "maxwell" else None
    P.rhs(p.directions[0], pol, 1, b)
    J = torch.zeros_like(b)
    md = vie.VIE_SOLVE_MIXED if mode == "mixed" else vie.VIE_SOLVE_FP64
    st, info = P.solve(b, J, tol=1e-10, restart=50, mode=md, check_fp64=True)
    assert st == vie.VIE_OK and info.rel_residual <= 1e-10
    assert 0.0 <= info.rel_residual_fp64 <= 1.5e-10
    Jo, oi = solvers.gmres(op.apply, op.rhs(p.directions[0], pol), tol=1e-12, restart=60, maxiter=600)
    assert oi["converged"]
    assert rel(J.cpu().numpy(), Jo) <= 1e-8


def test_oscillatory_medium_solve_bluestein(vie):
    """The first experiment's problem (reduced Maxwell, oscillatory isotropic eps,
    E^in = (0, 0, exp(i w x)) on [0,1]^3) at n = 26 with w = 40: the mixed solve
    through Bluestein transforms (2n = 52, 3n = 78) equals the oracle's FP64 GMRES."""
    import torch

    n = 26
    p = vi.oscillatory_problem(n, 40.0)
    P = vie.Problem("maxwell", n, p.lo, p.hi, p.omega, eps_dev(p), None)
    b = torch.empty((3, n, n, n), dtype=torch.complex128, device="cuda:0")
    P.rhs(p.directions[0], p.polarisations[0], 1, b)
    J = torch.zeros_like(b)
    st, info = P.solve(b, J, tol=1e-10, restart=50, mode=vie.VIE_SOLVE_MIXED)
    assert st == vie.VIE_OK and info.rel_residual <= 1e-10
    op = operators.OracleProblem.from_problem(p)
    bo = op.rhs(p.directions[0], p.polarisations[0])
    assert rel(b.cpu().numpy(), bo) <= 1e-13
    Jo, oi = solvers.gmres(op.apply, bo, tol=1e-12, restart=60, maxiter=600)
    assert oi["converged"]
    assert rel(J.cpu().numpy(), Jo) <= 1e-8
    P.close()
