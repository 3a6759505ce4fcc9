"""Double-word (VIE_DF64) operator apply and the mixed solve's residuals.

VIE_DF64 takes FP64 vectors and computes in double-word arithmetic (two FP32
values per real, about 48 significant bits).  Its result must match the FP64
oracle as closely as the native FP64 apply does: the per-operation error bound
of the double-word add and multiply is a few u^2 with u = 2^-24 (about 1e-14),
which the FFT's log-depth accumulation keeps far below the 1e-12 bar of the
FP64 parity tests.  A plain FP32 apply misses that bar by five orders.
"""
import numpy as np
import pytest

import vie_inputs as vi
from gpu_common import eps_dev, mu_dev, rel, to_dev, vie  # noqa: F401
from oracle import operators, solvers

pytestmark = pytest.mark.gpu

CASES = [
    ("laplace", 12, 0.0, False),
    ("laplace", 32, 0.0, False),
    ("helmholtz", 24, 4.0, False),
    ("helmholtz", 64, 4.0, False),
    ("maxwell", 12, 2.0, True),
    ("maxwell", 16, 3.0, False),
]


def make_problem(kind, n, wavelengths, with_mu, seed=0):
    if kind == "laplace":
        return vi.laplace_bump_problem(n=n, seed=seed)
    if kind == "helmholtz":
        return vi.helmholtz_problem(n=n, wavelengths=wavelengths, seed=seed)
    return vi.maxwell_problem(n=n, wavelengths=wavelengths, with_mu=with_mu, seed=seed)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}-mu{int(c[3])}")
def test_apply_df64_matches_oracle(vie, case):
    import torch

    p = make_problem(case[0], case[1], case[2], case[3])
    op = operators.OracleProblem.from_problem(p)
    P = vie.Problem(case[0], p.n, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
    try:
        x = vi.random_field(p.n, op.ncomp, 3)[0]
        xd = to_dev(x)
        yd = torch.empty_like(xd)
        P.apply(xd, yd, vie.VIE_DF64)
        torch.cuda.synchronize()
        assert rel(yd.cpu().numpy(), op.apply(x)) <= 1e-12
    finally:
        P.close()


def test_apply_df64_full_size_and_batched(vie):
    """At the 128^3 Helmholtz workload the double-word apply equals the FP64 one
    to FP64-level accuracy; two right-hand sides in one call equal two calls."""
    import torch

    p = vi.helmholtz_problem(n=128, wavelengths=4.0, seed=0)
    P = vie.Problem("helmholtz", 128, p.lo, p.hi, p.omega, eps_dev(p))
    try:
        g = torch.Generator(device="cuda:0")
        g.manual_seed(5)
        x = torch.randn((2, 3, 128, 128, 128), dtype=torch.complex128, device="cuda:0", generator=g)
        y64 = torch.empty_like(x[0])
        P.apply(x[0], y64, vie.VIE_FP64)
        ydf = torch.empty_like(x)
        P.apply(x, ydf, vie.VIE_DF64, nrhs=2)
        y1 = torch.empty_like(x[1])
        P.apply(x[1], y1, vie.VIE_DF64)
        torch.cuda.synchronize()
        assert rel(ydf[0].cpu().numpy(), y64.cpu().numpy()) <= 1e-12
        assert torch.equal(ydf[1], y1)
        assert P.tune(vie.VIE_DF64) == -1  # one fixed double-word schedule: nothing to tune
    finally:
        P.close()


@pytest.mark.parametrize("case", [("helmholtz", 24, 4.0, False), ("maxwell", 12, 2.0, True)],
                         ids=lambda c: f"{c[0]}-{c[1]}-mu{int(c[3])}")
def test_mixed_solve_with_double_word_residuals(vie, monkeypatch, case):
    """The mixed solve with double-word residuals (the default) and with native
    FP64 residuals both reach the oracle's solution, and the native FP64
    residual of the double-word run's answer meets the tolerance."""
    import torch

    p = make_problem(*case)
    op = operators.OracleProblem.from_problem(p)
    P = vie.Problem(case[0], p.n, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
    try:
        d = p.directions[0]
        pol = p.polarisations[0] if p.kind == "maxwell" else None
        b = torch.empty((op.ncomp, p.n, p.n, p.n), dtype=torch.complex128, device="cuda:0")
        P.rhs(d, pol, 1, b)
        Jo, _ = solvers.gmres(op.apply, op.rhs(d, pol), tol=1e-13, restart=60)
        sols = []
        for native in (False, True):
            if native:
                monkeypatch.setenv("VIE_RESIDUAL_FP64", "1")
            else:
                monkeypatch.delenv("VIE_RESIDUAL_FP64", raising=False)
            J = torch.zeros_like(b)
            st, info = P.solve(b, J, tol=1e-10, restart=40, mode=vie.VIE_SOLVE_MIXED, inner_tol=1e-5, max_outer=30)
            assert info.rel_residual <= 1e-10
            assert rel(J.cpu().numpy(), Jo) <= 1e-8
            sols.append(J)
        monkeypatch.delenv("VIE_RESIDUAL_FP64", raising=False)
        r = torch.empty_like(b)
        P.apply(sols[0], r, vie.VIE_FP64)
        torch.cuda.synchronize()
        true_res = float(torch.linalg.vector_norm(r - b) / torch.linalg.vector_norm(b))
        assert true_res <= 1.5e-10
    finally:
        P.close()


def test_apply_df64_maxwell_128_fast_path(vie):
    """Maxwell with mu at 128^3 (2n = 256: the register-resident double-word
    passes and 6x6 z pass) equals the FP64 apply to FP64-level accuracy."""
    import torch

    p = vi.maxwell_problem(n=128, wavelengths=5.0, with_mu=True, seed=1)
    P = vie.Problem("maxwell", 128, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
    try:
        g = torch.Generator(device="cuda:0")
        g.manual_seed(6)
        x = torch.randn((6, 128, 128, 128), dtype=torch.complex128, device="cuda:0", generator=g)
        y64 = torch.empty_like(x)
        ydf = torch.empty_like(x)
        P.apply(x, y64, vie.VIE_FP64)
        P.apply(x, ydf, vie.VIE_DF64)
        torch.cuda.synchronize()
        assert rel(ydf.cpu().numpy(), y64.cpu().numpy()) <= 1e-12
    finally:
        P.close()
