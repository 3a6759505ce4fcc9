"""GPU parity of whole solves at the grid sizes the register-resident kernels run.

The generic-kernel sizes (2n = 24, 48) are covered in test_gpu_parity.py; here
every solve runs the fast path: 2n = 64 and 128 (n = 32, 64) for single and
batched mixed solves, and 2n = 256 (n = 128, the benchmarked Helmholtz
workload) for one mixed solve whose refinement residuals take the double-word
apply (the default residual path; its register-resident kernels exist only at
2n = 256).  The oracle solves the same discrete system with its own FP64
GMRES (Sec. 1 / Sec. 6) on the host cores.

Tolerance: the mixed solve stops at a relative residual of 1e-10; the
operators are second kind (Eqs. (eq:intLap), (eq:intH), (eq:intM)) with
condition numbers of order 10 on these media, so the solution error is about
1e-9; the bar is 1e-8, tighter than the 1e-6 bound stated for mixed paths.
"""
import numpy as np
import pytest

import vie_inputs as vi
from oracle import operators, solvers

from gpu_common import eps_dev, mu_dev, rel, vie  # noqa: F401

pytestmark = pytest.mark.gpu

FAST_CASES = [
    ("helmholtz", 32, 3.0, False),
    ("helmholtz", 64, 4.0, False),
    ("laplace", 64, 0.0, False),
    ("maxwell", 32, 2.0, True),
    ("maxwell", 64, 3.0, False),
]


def _problem(kind, n, wl, with_mu, seed, ndirs=1, npol=1):
    if kind == "laplace":
        return vi.laplace_bump_problem(n=n, seed=seed)
    if kind == "helmholtz":
        return vi.helmholtz_problem(n=n, wavelengths=wl, nrhs=ndirs, seed=seed)
    return vi.maxwell_problem(n=n, wavelengths=wl, ndirs=ndirs, npol=npol, with_mu=with_mu, seed=seed)


def _oracle_solution(op, p, r):
    pol = p.polarisations[r] if p.kind == "maxwell" else None
    b = op.rhs(p.directions[r], pol)
    J, info = solvers.gmres(op.apply, b, tol=1e-12, restart=60, maxiter=600)
    assert info["converged"]
    return J


@pytest.mark.parametrize("case", FAST_CASES, ids=lambda c: f"{c[0]}-{c[1]}-mu{int(c[3])}")
def test_mixed_solve_fast_sizes(vie, case):
    """Mixed solve (FP32 register-resident applies, double-word residuals) = oracle FP64 GMRES."""
    import torch

    kind, n, wl, with_mu = case
    p = _problem(kind, n, wl, with_mu, seed=3)
    P = vie.Problem(kind, n, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
    assert P.tune(vie.VIE_FP32) >= 0, "this size must take a register-resident z pass"
    b = torch.empty((P.ncomp, n, n, n), dtype=torch.complex128, device="cuda:0")
    pol = p.polarisations[0] if kind == "maxwell" else None
    P.rhs(p.directions[0], pol, 1, b)
    J = torch.zeros_like(b)
    st, info = P.solve(b, J, tol=1e-10, restart=50, mode=vie.VIE_SOLVE_MIXED, inner_tol=1e-5, check_fp64=True)
    assert st == vie.VIE_OK and info.rel_residual <= 1e-10
    assert info.applies_fp32 > 0 and info.applies_fp64 >= 1
    # the native FP64 residual of the returned iterate agrees with the double-word one
    assert 0.0 <= info.rel_residual_fp64 <= 1.5e-10
    assert info.t_precompute > 0.0
    op = operators.OracleProblem.from_problem(p)
    Jo = _oracle_solution(op, p, 0)
    assert rel(J.cpu().numpy(), Jo) <= 1e-8, (kind, n)
    P.close()


@pytest.mark.parametrize("kind,n,wl,with_mu,ndirs,npol", [("maxwell", 32, 2.0, True, 2, 2),
                                                          ("helmholtz", 64, 3.0, False, 4, 1)],
                         ids=["maxwell-32-mu1-x4", "helmholtz-64-x4"])
def test_batched_mixed_solve_fast_sizes(vie, kind, n, wl, with_mu, ndirs, npol):
    """Four right-hand sides in one lockstep group at a register-resident size; each = oracle."""
    import torch

    p = _problem(kind, n, wl, with_mu, seed=6, ndirs=ndirs, npol=npol)
    P = vie.Problem(kind, n, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
    nr = p.nrhs
    assert nr == 4
    b = torch.empty((nr, P.ncomp, n, n, n), dtype=torch.complex128, device="cuda:0")
    P.rhs(p.directions, p.polarisations if kind == "maxwell" else None, nr, b)
    J = torch.zeros_like(b)
    st, info = P.solve(b, J, tol=1e-10, restart=40, mode=vie.VIE_SOLVE_MIXED, nrhs=nr)
    assert st == vie.VIE_OK and info.rel_residual <= 1e-10
    op = operators.OracleProblem.from_problem(p)
    for r in range(nr):
        Jo = _oracle_solution(op, p, r)
        assert rel(J[r].cpu().numpy(), Jo) <= 1e-8, r
    P.close()


def test_mixed_solve_128_double_word_residuals(vie, monkeypatch):
    """The benchmarked Helmholtz 128^3 workload (4 wavelengths, multi-bump medium):
    the mixed solve with its default residual path (double-word apply, register-
    resident at 2n = 256) reaches the oracle's FP64 solution."""
    import torch

    monkeypatch.delenv("VIE_RESIDUAL_FP64", raising=False)
    n = 128
    p = vi.helmholtz_problem(n=n, wavelengths=4.0, seed=0)
    P = vie.Problem("helmholtz", n, p.lo, p.hi, p.omega, eps_dev(p))
    b = torch.empty((3, n, n, n), dtype=torch.complex128, device="cuda:0")
    P.rhs(p.directions[0], None, 1, b)
    J = torch.zeros_like(b)
    st, info = P.solve(b, J, tol=1e-10, restart=50, mode=vie.VIE_SOLVE_MIXED, inner_tol=1e-5)
    assert st == vie.VIE_OK and info.rel_residual <= 1e-10
    assert info.applies_fp64 >= 1  # refinement residuals were computed (double-word apply)
    Jg = J.cpu().numpy()
    del b, J
    torch.cuda.empty_cache()
    op = operators.OracleProblem.from_problem(p)
    Jo = _oracle_solution(op, p, 0)
    assert rel(Jg, Jo) <= 1e-8
    P.close()


@pytest.mark.parametrize("kind,n,mode", [("laplace", 32, "mixed"), ("helmholtz", 24, "fp64"), ("maxwell", 16, "mixed")])
def test_graph_replayed_steps_equal_direct_launches(vie, monkeypatch, kind, n, mode):
    """From the second GMRES cycle with an unchanged layout, single-RHS Arnoldi steps
    are replayed as CUDA graphs; repeated solves through the replays give the
    direct-launch answer bit for bit (same kernels, same order) and the oracle's."""
    import torch

    md = vie.VIE_SOLVE_MIXED if mode == "mixed" else vie.VIE_SOLVE_FP64
    p = _problem(kind, n, 2.0, kind == "maxwell", seed=4)
    outs = {}
    for graphs in ("0", "1"):
        monkeypatch.setenv("VIE_GRAPHS", graphs)
        P = vie.Problem(kind, n, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
        b = torch.empty((P.ncomp, n, n, n), dtype=torch.complex128, device="cuda:0")
        P.rhs(p.directions[0], p.polarisations[0] if kind == "maxwell" else None, 1, b)
        res = []
        for _ in range(3):  # later solves run their cycles from captured graphs
            J = torch.zeros_like(b)
            st, info = P.solve(b, J, tol=1e-10, restart=8 if mode == "fp64" else 40, max_outer=60, mode=md)
            assert st == vie.VIE_OK and info.rel_residual <= 1e-10
            res.append(J.cpu().numpy())
        outs[graphs] = res
        P.close()
    for a, g in zip(outs["0"], outs["1"]):
        assert np.array_equal(a, g)
    op = operators.OracleProblem.from_problem(p)
    assert rel(outs["1"][-1], _oracle_solution(op, p, 0)) <= 1e-8


@pytest.mark.parametrize("kind,n,wl", [("helmholtz", 64, 4.0), ("laplace", 32, 0.0)])
def test_fp32_updated_residual_is_certified(vie, monkeypatch, kind, n, wl):
    """At tol = 1e-8 the residual after a small refinement correction d is updated
    as r -= A_32 d (FP32 apply) when the bound on that apply's error is within half
    the tolerance; the reported residual includes the bound, so the native FP64
    residual of the answer is below it.  With VIE_RESIDUAL_UPDATE=0 every residual
    is a double-word apply; both answers agree with the oracle."""
    import torch

    p = _problem(kind, n, wl, False, seed=8)
    op = operators.OracleProblem.from_problem(p)
    Jo = _oracle_solution(op, p, 0)
    res = {}
    for upd in ("1", "0"):
        monkeypatch.setenv("VIE_RESIDUAL_UPDATE", upd)
        P = vie.Problem(kind, n, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
        b = torch.empty((P.ncomp, n, n, n), dtype=torch.complex128, device="cuda:0")
        P.rhs(p.directions[0], None, 1, b)
        J = torch.zeros_like(b)
        st, info = P.solve(b, J, tol=1e-8, restart=50, mode=vie.VIE_SOLVE_MIXED, check_fp64=True)
        assert st == vie.VIE_OK and info.rel_residual <= 1e-8
        assert 0.0 <= info.rel_residual_fp64 <= info.rel_residual * 1.0001 + 1e-14
        assert rel(J.cpu().numpy(), Jo) <= 1e-6
        res[upd] = info
        P.close()
    # the updated path replaces double-word residual applies by FP32 ones
    assert res["1"].applies_fp64 < res["0"].applies_fp64
