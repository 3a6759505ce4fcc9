"""GPU parity: the CUDA library (through the C ABI) against the FP64 CPU oracle.

Tolerances (relative L2 over all components):
* FP64 apply / rhs / scattered field: 1e-12 (both sides compute the same
  discrete convolution in FP64; they differ only in rounding order).
* FP32 apply: 2e-5.  Each FFT stage adds ~eps_32 = 6e-8 relative error; a
  pruned forward plus inverse 3D transform on (2n)^3 has 2 log2((2n)^3) ~ 50
  butterfly levels at 2n = 256, i.e. ~3e-6 -- the tolerance leaves a 6x margin.
* FP64 solve: 1e-10 (the parity bound for FP64 paths); mixed solve: the bound
  after refinement is 1e-6, tested here at a tighter 1e-8.
"""
import math

import numpy as np
import pytest

import vie_inputs as vi
from oracle import operators, solvers

from gpu_common import eps_dev, mu_dev, rel, to_dev, vie  # noqa: F401

pytestmark = pytest.mark.gpu

CASES = [
    ("laplace", 8, 0.0, False),
    ("laplace", 12, 0.0, False),
    ("laplace", 32, 0.0, False),
    ("helmholtz", 8, 2.0, False),
    ("helmholtz", 24, 4.0, False),
    ("maxwell", 8, 1.5, False),
    ("maxwell", 12, 2.0, True),
    ("maxwell", 16, 3.0, True),
]


def make_problem(kind, n, wavelengths, with_mu, seed=0):
    if kind == "laplace":
        return vi.laplace_bump_problem(n=n, seed=seed)
    if kind == "helmholtz":
        return vi.helmholtz_problem(n=n, wavelengths=wavelengths, seed=seed)
    return vi.maxwell_problem(n=n, wavelengths=wavelengths, with_mu=with_mu, seed=seed)


_cache = {}


def setup(vie, kind, n, wl, with_mu):
    key = (kind, n, wl, with_mu)
    if key not in _cache:
        p = make_problem(kind, n, wl, with_mu)
        P = vie.Problem(kind, n, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
        op = operators.OracleProblem.from_problem(p)
        _cache[key] = (p, P, op)
    return _cache[key]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}-mu{int(c[3])}")
def test_apply_fp64(vie, case):
    import torch

    p, P, op = setup(vie, *case)
    x = vi.random_field(p.n, op.ncomp, 1)[0]
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    P.apply(xd, yd, vie.VIE_FP64)
    torch.cuda.synchronize()
    assert rel(yd.cpu().numpy(), op.apply(x)) <= 1e-12


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}-mu{int(c[3])}")
def test_apply_fp32(vie, case):
    import torch

    p, P, op = setup(vie, *case)
    x = vi.random_field(p.n, op.ncomp, 2)[0]
    xd = to_dev(x, torch.complex64)
    yd = torch.empty_like(xd)
    P.apply(xd, yd, vie.VIE_FP32)
    torch.cuda.synchronize()
    assert rel(yd.cpu().numpy(), op.apply(x.astype(np.complex64).astype(np.complex128))) <= 2e-5


def test_apply_batched_equals_single(vie):
    import torch

    p, P, op = setup(vie, "helmholtz", 24, 4.0, False)
    x = vi.random_field(p.n, 3, 3, nrhs=3)
    xd = to_dev(x)
    yb = torch.empty_like(xd)
    P.apply(xd, yb, vie.VIE_FP64, nrhs=3)
    for r in range(3):
        ys = torch.empty_like(xd[r])
        P.apply(xd[r].contiguous(), ys, vie.VIE_FP64)
        torch.cuda.synchronize()
        assert torch.equal(ys, yb[r])


@pytest.mark.parametrize("case", CASES[::2] + [CASES[6]], ids=lambda c: f"{c[0]}-{c[1]}-mu{int(c[3])}")
def test_rhs(vie, case):
    import torch

    p, P, op = setup(vie, *case)
    out = torch.empty((op.ncomp, p.n, p.n, p.n), dtype=torch.complex128, device="cuda:0")
    d = p.directions[0]
    pol = p.polarisations[0] if p.kind == "maxwell" else None
    P.rhs(d, pol, 1, out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), op.rhs(d, pol)) <= 1e-13


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}-mu{int(c[3])}")
def test_scattered_field(vie, case):
    import torch

    p, P, op = setup(vie, *case)
    x = vi.random_field(p.n, op.ncomp, 4)[0]
    cout = 1 if p.kind != "maxwell" else 6
    out = torch.empty((cout, p.n, p.n, p.n), dtype=torch.complex128, device="cuda:0")
    P.eval_scattered(to_dev(x), out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), op.scattered(x)) <= 1e-12


@pytest.mark.parametrize("case", [("laplace", 32, 0.0, False), ("helmholtz", 24, 4.0, False),
                                  ("maxwell", 16, 3.0, True)], ids=lambda c: f"{c[0]}-{c[1]}-mu{int(c[3])}")
def test_scattered_field_batched_equals_single(vie, case):
    """Two densities in one vie_eval_scattered call give, bit for bit, the fields of two
    single calls (n = 32 runs the register-resident kernels, 24 and 16 the generic ones)."""
    import torch

    p, P, op = setup(vie, *case)
    x = vi.random_field(p.n, op.ncomp, 5, nrhs=2)
    cout = 1 if p.kind != "maxwell" else 6
    xd = to_dev(x)
    out = torch.empty((2, cout, p.n, p.n, p.n), dtype=torch.complex128, device="cuda:0")
    P.eval_scattered(xd, out, nrhs=2)
    for r in range(2):
        single = torch.empty_like(out[r])
        P.eval_scattered(xd[r].contiguous(), single)
        torch.cuda.synchronize()
        assert torch.equal(single, out[r])
    assert rel(out[1].cpu().numpy(), op.scattered(x[1])) <= 1e-12


@pytest.mark.parametrize("kind,n", [("laplace", 12), ("helmholtz", 32), ("maxwell", 16)])
def test_vacuum_operator_is_identity(vie, kind, n):
    """No scatterer (eps = I, and mu = I given explicitly for Maxwell): H = 0, so the
    apply returns its input (exactly in FP64 and FP32; the double-word form holds ~48
    bits), the right-hand side is zero and the solve returns J = 0.  n = 32 runs the
    register-resident kernels."""
    import torch

    eye = to_dev(vi.identity_field(n).reshape(9, -1))
    P = vie.Problem(kind, n, -1.0, 1.0, 0.0 if kind == "laplace" else 2.0, eye, eye if kind == "maxwell" else None)
    try:
        c = P.ncomp
        x = vi.random_field(n, c, 19)[0]
        for prec, dt in ((vie.VIE_FP64, torch.complex128), (vie.VIE_FP32, torch.complex64),
                         (vie.VIE_DF64, torch.complex128)):
            xd = to_dev(x, dt)
            yd = torch.empty_like(xd)
            P.apply(xd, yd, prec)
            torch.cuda.synchronize()
            if prec == vie.VIE_DF64:
                assert rel(yd.cpu().numpy(), x) <= 1e-14
            else:
                assert torch.equal(yd, xd), prec
        b = torch.empty((c, n, n, n), dtype=torch.complex128, device="cuda:0")
        P.rhs(np.array([0.0, 0.6, 0.8]), np.array([1.0, 0.0, 0.0]) if kind == "maxwell" else None, 1, b)
        torch.cuda.synchronize()
        assert torch.count_nonzero(b) == 0
        J = torch.ones_like(b)
        P.solve(b, J)
        assert torch.count_nonzero(J) == 0
    finally:
        P.close()


@pytest.mark.parametrize("mode", ["fp64", "mixed", "bicgstab"])
def test_solve_from_nonzero_initial_guess(vie, mode):
    """A non-zero initial guess -- the solution perturbed by 1e-3, and a random vector
    ten times its size -- converges to the oracle's solution; the near guess takes
    fewer applies than a zero start (its residual is computed, not assumed to be b)."""
    import torch

    p, P, op = setup(vie, "helmholtz", 24, 4.0, False)
    m = {"fp64": vie.VIE_SOLVE_FP64, "mixed": vie.VIE_SOLVE_MIXED, "bicgstab": vie.VIE_SOLVE_BICGSTAB}[mode]
    d = p.directions[0]
    b = torch.empty((3, 24, 24, 24), dtype=torch.complex128, device="cuda:0")
    P.rhs(d, None, 1, b)
    Jo, _ = solvers.gmres(op.apply, op.rhs(d), tol=1e-13, restart=60)
    noise = vi.random_field(24, 3, 17)[0]
    scale = np.linalg.norm(Jo) / np.linalg.norm(noise)
    applies = []
    for J0 in (np.zeros_like(Jo), Jo + 1e-3 * scale * noise, 10 * scale * noise):
        J = to_dev(J0)
        st, info = P.solve(b, J, tol=1e-10, restart=40, mode=m, max_outer=30, max_inner=2000)
        assert info.rel_residual <= 1e-10
        assert rel(J.cpu().numpy(), Jo) <= 1e-8
        applies.append(info.applies_fp32 + info.applies_fp64)
    assert applies[1] < applies[0]


def test_solve_fp64_laplace_32(vie):
    """Config-1 workload: anisotropic Laplace bump, 32^3, GMRES to 1e-10 (FP64)."""
    import torch

    p, P, op = setup(vie, "laplace", 32, 0.0, False)
    b = torch.empty((3, 32, 32, 32), dtype=torch.complex128, device="cuda:0")
    P.rhs(p.directions[0], None, 1, b)
    J = torch.zeros_like(b)
    st, info = P.solve(b, J, tol=1e-12, restart=50, mode=vie.VIE_SOLVE_FP64)
    Jo, io = solvers.gmres(op.apply, op.rhs(p.directions[0]), tol=1e-13, restart=50)
    assert info.rel_residual <= 1e-12
    assert rel(J.cpu().numpy(), Jo) <= 1e-10


def test_solve_fp64_laplace_dense_8(vie):
    import torch

    p, P, op = setup(vie, "laplace", 8, 0.0, False)
    b = torch.empty((3, 8, 8, 8), dtype=torch.complex128, device="cuda:0")
    P.rhs(p.directions[0], None, 1, b)
    J = torch.zeros_like(b)
    P.solve(b, J, tol=1e-13, restart=60, mode=vie.VIE_SOLVE_FP64)
    Jo = solvers.dense_solve(op.apply, op.rhs(p.directions[0]))
    assert rel(J.cpu().numpy(), Jo) <= 1e-10


@pytest.mark.parametrize("case", [CASES[4], CASES[6]], ids=lambda c: f"{c[0]}-{c[1]}-mu{int(c[3])}")
def test_solve_mixed(vie, case):
    import torch

    p, P, op = setup(vie, *case)
    d = p.directions[0]
    pol = p.polarisations[0] if p.kind == "maxwell" else None
    b = torch.empty((op.ncomp, p.n, p.n, p.n), dtype=torch.complex128, device="cuda:0")
    P.rhs(d, pol, 1, b)
    J = torch.zeros_like(b)
    st, info = P.solve(b, J, tol=1e-10, restart=40, mode=vie.VIE_SOLVE_MIXED, inner_tol=1e-5, max_outer=30)
    Jo, _ = solvers.gmres(op.apply, op.rhs(d, pol), tol=1e-13, restart=60)
    assert info.rel_residual <= 1e-10
    assert info.applies_fp32 > info.applies_fp64
    assert rel(J.cpu().numpy(), Jo) <= 1e-8


def test_solve_fp64_helmholtz_multi_rhs(vie):
    import torch

    p = vi.helmholtz_problem(n=12, wavelengths=2.0, nrhs=2, seed=4)
    P = vie.Problem("helmholtz", 12, p.lo, p.hi, p.omega, eps_dev(p))
    op = operators.OracleProblem.from_problem(p)
    b = torch.empty((2, 3, 12, 12, 12), dtype=torch.complex128, device="cuda:0")
    P.rhs(p.directions, None, 2, b)
    J = torch.zeros_like(b)
    st, info = P.solve(b, J, tol=1e-12, restart=30, mode=vie.VIE_SOLVE_FP64, nrhs=2)
    for r in range(2):
        Jo, _ = solvers.gmres(op.apply, op.rhs(p.directions[r]), tol=1e-13, restart=60)
        assert rel(J[r].cpu().numpy(), Jo) <= 1e-10


def test_invalid_arguments(vie):
    import torch

    p = vi.laplace_bump_problem(n=8)
    e = eps_dev(p)
    for bad in [dict(n=3), dict(n=-4), dict(n=513), dict(lo=1.0, hi=1.0), dict(omega=-1.0)]:
        kw = dict(kind=vie.VIE_LAPLACE, n=8, lo=-1.0, hi=1.0, omega=0.0)
        kw.update(bad)
        with pytest.raises(vie.VieError) as ei:
            vie.vie_problem_create(kw["kind"], kw["n"], kw["lo"], kw["hi"], kw["omega"], e)
        assert ei.value.status == vie.VIE_EINVAL
    asym = p.eps.copy()
    asym[0, 1] += 0.1
    with pytest.raises(vie.VieError) as ei:
        vie.vie_problem_create(vie.VIE_LAPLACE, 8, -1.0, 1.0, 0.0, to_dev(asym.reshape(9, -1)))
    assert ei.value.status == vie.VIE_EINVAL
    with pytest.raises(vie.VieError):
        vie.vie_problem_create(vie.VIE_HELMHOLTZ, 8, -1.0, 1.0, 0.0, e)
    P = vie.Problem("laplace", 8, -1.0, 1.0, 0.0, e)
    x = torch.zeros((3, 8, 8, 8), dtype=torch.complex128, device="cuda:0")
    with pytest.raises(vie.VieError):
        vie.vie_apply(P.handle, x, x, vie.VIE_FP64)
    with pytest.raises(vie.VieError):
        vie.vie_apply(P.handle, x, torch.empty_like(x), 7)
    # plane waves: unit directions, transverse polarisations (Laplace's d is E0: any vector)
    b3 = torch.empty((3, 8, 8, 8), dtype=torch.complex128, device="cuda:0")
    P.rhs(np.array([0.0, 0.0, 2.5]), None, 1, b3)
    for kind in ("helmholtz", "maxwell"):
        Q = vie.Problem(kind, 8, -1.0, 1.0, 2.0, e)
        pol = np.array([1.0, 0.0, 0.0]) if kind == "maxwell" else None
        Q.rhs(np.array([0.0, 0.6, 0.8]), pol, 1, b3)
        for dd, pp in ((np.array([0.0, 0.0, 2.0]), pol), (np.array([0.0, 0.0, np.nan]), pol)) + \
                (((np.array([0.0, 0.6, 0.8]), np.array([0.0, 1.0, 0.0])),) if kind == "maxwell" else ()):
            with pytest.raises(vie.VieError) as ei:
                Q.rhs(dd, pp, 1, b3)
            assert ei.value.status == vie.VIE_EINVAL
        Q.close()
    # a valid apply first: buffers that touch without sharing a byte are accepted
    N = 8 ** 3
    f32 = torch.zeros(2 * 3 * N, dtype=torch.complex64, device="cuda:0")
    vie.vie_apply(P.handle, f32[:3 * N].view(3, 8, 8, 8), f32[3 * N:].view(3, 8, 8, 8), vie.VIE_FP32)  # adjacent
    y = torch.empty_like(x)
    vie.vie_apply(P.handle, x, y, vie.VIE_FP64)
    torch.cuda.synchronize()
    # views one element apart share all but one element: every entry point refuses them
    buf = torch.zeros(3 * N + 1, dtype=torch.complex128, device="cuda:0")
    a, b = buf[:3 * N].view(3, 8, 8, 8), buf[1:].view(3, 8, 8, 8)
    for call in (lambda: vie.vie_apply(P.handle, a, b, vie.VIE_FP64),
                 lambda: vie.vie_solve(P.handle, a, b, vie.SolveOpts(1e-10, 20, 5, 100, 1e-5, vie.VIE_SOLVE_FP64, 1)),
                 lambda: vie.vie_eval_scattered(P.handle, a, buf[2 * N:3 * N].view(1, 8, 8, 8)),
                 # FP32 vectors: 8 bytes per value
                 lambda: vie.vie_apply(P.handle, f32[:3 * N].view(3, 8, 8, 8),
                                       f32[3 * N - 1:6 * N - 1].view(3, 8, 8, 8), vie.VIE_FP32)):
        with pytest.raises(vie.VieError) as ei:
            call()
        assert ei.value.status == vie.VIE_EINVAL


def test_smallest_grid_and_zero_input(vie):
    import torch

    p = vi.laplace_bump_problem(n=4)
    P = vie.Problem("laplace", 4, p.lo, p.hi, 0.0, eps_dev(p))
    op = operators.OracleProblem.from_problem(p)
    x = vi.random_field(4, 3, 9)[0]
    y = torch.empty((3, 4, 4, 4), dtype=torch.complex128, device="cuda:0")
    P.apply(to_dev(x), y, vie.VIE_FP64)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), op.apply(x)) <= 1e-12
    z = torch.zeros_like(y)
    P.apply(z, y, vie.VIE_FP64)
    torch.cuda.synchronize()
    assert torch.count_nonzero(y) == 0
    # a zero right-hand side solves to zero without iterating
    J = torch.ones_like(y)
    st, info = P.solve(z, J)
    assert torch.count_nonzero(J) == 0


def test_low_frequency_helmholtz_equals_laplace_inverse_eps(vie):
    """w -> 0: the Helmholtz operator with eps equals the Laplace operator with eps^-1 (GPU only)."""
    import torch

    n = 12
    # Laplace takes Re(eps): use a lossless medium so that eps^-1 is real
    p2 = vi.helmholtz_problem(n=n, wavelengths=1e-10, seed=2, lossless=True)
    Ph = vie.Problem("helmholtz", n, p2.lo, p2.hi, p2.omega, eps_dev(p2))
    Pl = vie.Problem("laplace", n, p2.lo, p2.hi, 0.0, to_dev(operators.inverse_field(p2.eps).reshape(9, -1)))
    x = to_dev(vi.random_field(n, 3, 5)[0])
    yh = torch.empty_like(x)
    yl = torch.empty_like(x)
    Ph.apply(x, yh, vie.VIE_FP64)
    Pl.apply(x, yl, vie.VIE_FP64)
    torch.cuda.synchronize()
    assert rel(yh.cpu().numpy(), yl.cpu().numpy()) <= 1e-12


@pytest.mark.slow
def test_full_size_helmholtz_128_fp32(vie):
    """The workload bench.py times (Helmholtz, 128^3, FP32 apply): every output against the oracle."""
    import torch

    p = vi.helmholtz_problem(n=128, wavelengths=4.0, seed=0)
    P = vie.Problem("helmholtz", 128, p.lo, p.hi, p.omega, eps_dev(p))
    x = vi.random_field(128, 3, 0)[0]
    xd = to_dev(x, torch.complex64)
    y32 = torch.empty_like(xd)
    P.apply(xd, y32, vie.VIE_FP32)
    y64 = torch.empty((3, 128, 128, 128), dtype=torch.complex128, device="cuda:0")
    P.apply(xd.to(torch.complex128), y64, vie.VIE_FP64)
    torch.cuda.synchronize()
    op = operators.OracleProblem.from_problem(p)
    yo = op.apply(x.astype(np.complex64).astype(np.complex128))
    assert rel(y64.cpu().numpy(), yo) <= 1e-12
    assert rel(y32.cpu().numpy(), yo) <= 2e-5


def gaussian_fields(n, alpha=36.0):
    import vie_inputs as vi_

    Z, Y, X = vi_.grid_coords(n, -1.0, 1.0)
    psi = np.exp(-alpha * (X * X + Y * Y + Z * Z))
    grad = np.stack([-2 * alpha * X * psi, -2 * alpha * Y * psi, -2 * alpha * Z * psi]).astype(np.complex128)
    curl = np.stack([-2 * alpha * Y * psi, 2 * alpha * X * psi, 0 * psi]).astype(np.complex128)
    return grad, curl


@pytest.mark.parametrize("n", [64, 128, 256])
@pytest.mark.parametrize("kind", ["laplace", "helmholtz"])
def test_lemma2_eigenfields_at_full_size(vie, n, kind):
    """Property that holds at any size (Lemma 2): with a constant isotropic eps = e I
    (H = h I, h = (e-1)/(e+1)) the operator maps grad psi and curl P of a resolved
    Gaussian to multiples of themselves:
      Laplace   A grad psi = (1 + h) grad psi,  A curl P = (1 - h) curl P;
      Helmholtz A curl P = (1 + h) curl P (for every w).
    Checks every pass, the kernels and the H epilogue at the sizes the configurations use."""
    import torch

    e = 3.0
    h = (e - 1) / (e + 1)
    eps = np.zeros((9, n, n, n), np.complex128)
    for a in range(3):
        eps[4 * a] = e
    omega = 0.0 if kind == "laplace" else 4 * math.pi
    P = vie.Problem(kind, n, -1.0, 1.0, omega, to_dev(eps))
    del eps
    grad, curl = gaussian_fields(n)
    cases = [(curl, (1 - h) if kind == "laplace" else (1 + h))]
    if kind == "laplace":
        cases.append((grad, 1 + h))
    for field, lam in cases:
        for prec, dt, tol in ((vie.VIE_FP64, torch.complex128, 1e-11), (vie.VIE_FP32, torch.complex64, 2e-5)):
            xd = to_dev(field, dt)
            yd = torch.empty_like(xd)
            P.apply(xd, yd, prec)
            torch.cuda.synchronize()
            got = yd.to(torch.complex128)
            ref = lam * xd.to(torch.complex128)
            err = float(torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref))
            assert err <= tol, (kind, n, prec, err)
    P.close()


@pytest.mark.parametrize("n", [32, 64])
def test_fast_and_generic_paths_agree_with_oracle(vie, n, monkeypatch):
    """Both the register-resident kernels (2n in {64,128,256,512}) and the generic
    shared-memory Stockham kernels reproduce the oracle."""
    import torch

    p = vi.helmholtz_problem(n=n, wavelengths=3.0, seed=5)
    op = operators.OracleProblem.from_problem(p)
    x = vi.random_field(n, 3, 6)[0]
    yo = op.apply(x)
    outs = []
    for generic in (False, True):
        if generic:
            monkeypatch.setenv("VIE_GENERIC_FFT", "1")
        P = vie.Problem("helmholtz", n, p.lo, p.hi, p.omega, eps_dev(p))
        xd = to_dev(x)
        yd = torch.empty_like(xd)
        P.apply(xd, yd, vie.VIE_FP64)
        torch.cuda.synchronize()
        outs.append(yd.cpu().numpy())
        P.close()
    monkeypatch.delenv("VIE_GENERIC_FFT", raising=False)
    for y in outs:
        assert rel(y, yo) <= 1e-12


@pytest.mark.parametrize("variant", list(range(19)))
@pytest.mark.parametrize("kind,n,mu", [("helmholtz", 32, False), ("maxwell", 32, True), ("helmholtz", 64, False),
                                       ("helmholtz", 48, False), ("maxwell", 48, True), ("laplace", 96, False),
                                       ("helmholtz", 128, False)])
def test_every_zpass_variant_matches_oracle(vie, monkeypatch, variant, kind, n, mu):
    """Each schedule the autotuner can pick (forced with VIE_P3_VARIANT) reproduces the oracle
    in every precision it applies to (the lane-pair variants 4-6 are FP32 only)."""
    import torch

    assert vie.P3_VARIANTS == 19
    p = make_problem(kind, n, 2.0, mu, seed=8)
    op = operators.OracleProblem.from_problem(p)
    x = vi.random_field(n, op.ncomp, 10)[0]
    monkeypatch.setenv("VIE_P3_VARIANT", str(variant))
    P = vie.Problem(kind, n, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
    applied = 0
    try:
        for prec, dt, tol in ((vie.VIE_FP64, torch.complex128, 1e-12), (vie.VIE_FP32, torch.complex64, 2e-5)):
            xd = to_dev(x, dt)
            yd = torch.empty_like(xd)
            try:
                P.apply(xd, yd, prec)
            except vie.VieError as e:
                assert e.status == vie.VIE_EINVAL
                continue
            torch.cuda.synchronize()
            xr = x if prec == vie.VIE_FP64 else x.astype(np.complex64).astype(np.complex128)
            assert rel(yd.cpu().numpy(), op.apply(xr)) <= tol
            assert P.tune(prec) == variant  # the forced schedule is the one that ran
            applied += 1
    finally:
        P.close()
        monkeypatch.delenv("VIE_P3_VARIANT", raising=False)
    if not applied:
        pytest.skip(f"variant {variant} does not apply to {kind} n={n}")


def test_zpass_variants_at_2n_512(vie, monkeypatch):
    """Maxwell with mu at 256^3 (2n = 512, the largest z-pass shapes): every
    variant that fits reproduces the FP64 apply of the same input in FP32; the
    FP64 path at this size is the one the smaller full-size tests pin to the
    oracle.  At least one mirror-group variant must apply here."""
    import torch

    n = 256
    p = vi.maxwell_problem(n=n, wavelengths=10.0, with_mu=True, seed=0)
    eps, mu = eps_dev(p), mu_dev(p)
    g = torch.Generator(device="cuda:0")
    g.manual_seed(3)
    x = torch.randn((6, n, n, n), dtype=torch.complex64, device="cuda:0", generator=g)
    y64 = torch.empty((6, n, n, n), dtype=torch.complex128, device="cuda:0")
    P = vie.Problem("maxwell", n, p.lo, p.hi, p.omega, eps, mu)
    P.apply(x.to(torch.complex128), y64, vie.VIE_FP64)
    P.close()
    ran = []
    for v in range(vie.P3_VARIANTS):
        monkeypatch.setenv("VIE_P3_VARIANT", str(v))
        P = vie.Problem("maxwell", n, p.lo, p.hi, p.omega, eps, mu)
        try:
            y32 = torch.empty_like(x)
            try:
                P.apply(x, y32, vie.VIE_FP32)
            except vie.VieError as e:
                assert e.status == vie.VIE_EINVAL
                continue
            torch.cuda.synchronize()
            assert P.tune(vie.VIE_FP32) == v
            err = float(torch.linalg.vector_norm(y32.to(torch.complex128) - y64) / torch.linalg.vector_norm(y64))
            assert err <= 2e-5, (v, err)
            ran.append(v)
        finally:
            P.close()
            monkeypatch.delenv("VIE_P3_VARIANT", raising=False)
    assert any(v in ran for v in (0, 1, 2)), ran
    assert all(v in ran for v in (15, 16, 17, 18)), ran  # the half-spectrum cluster z pass exists at this shape


@pytest.mark.parametrize("variant", [15, 16, 17, 18])
@pytest.mark.parametrize("kind", ["laplace", "helmholtz"])
def test_half_spectrum_zpass_eigenfields_at_2n_512(vie, monkeypatch, variant, kind):
    """The half-spectrum z pass (variants 15-18, 2n = 512 only: the even and odd
    frequencies of each z-line on the two CTAs of a cluster) on the Lemma 2
    eigenfields at 256^3, FP32: with eps = e I, Laplace maps grad psi to
    (1 + h) grad psi and curl P to (1 - h) curl P, Helmholtz curl P to (1 + h) curl P."""
    import torch

    n = 256
    e = 3.0
    h = (e - 1) / (e + 1)
    eps = np.zeros((9, n, n, n), np.complex128)
    for a in range(3):
        eps[4 * a] = e
    omega = 0.0 if kind == "laplace" else 4 * math.pi
    monkeypatch.setenv("VIE_P3_VARIANT", str(variant))
    P = vie.Problem(kind, n, -1.0, 1.0, omega, to_dev(eps))
    del eps
    try:
        grad, curl = gaussian_fields(n)
        cases = [(curl, (1 - h) if kind == "laplace" else (1 + h))]
        if kind == "laplace":
            cases.append((grad, 1 + h))
        for field, lam in cases:
            xd = to_dev(field, torch.complex64)
            yd = torch.empty_like(xd)
            P.apply(xd, yd, vie.VIE_FP32)
            torch.cuda.synchronize()
            assert P.tune(vie.VIE_FP32) == variant
            ref = lam * xd.to(torch.complex128)
            err = float(torch.linalg.vector_norm(yd.to(torch.complex128) - ref) / torch.linalg.vector_norm(ref))
            assert err <= 2e-5, (kind, variant, err)
    finally:
        P.close()
        monkeypatch.delenv("VIE_P3_VARIANT", raising=False)


def test_tune_entry_point(vie):
    p, P, op = setup(vie, "helmholtz", 24, 4.0, False)
    import paper_1805_04791_gb300 as m

    P2 = vie.Problem("helmholtz", 32, -1.0, 1.0, p.omega, eps_dev(vi.helmholtz_problem(n=32, wavelengths=4.0)))
    v32 = P2.tune(m.VIE_FP32)
    v64 = P2.tune(m.VIE_FP64)
    assert 0 <= v32 < vie.P3_VARIANTS and 0 <= v64 < 4
    assert P.tune(m.VIE_FP32) == -1  # 2n = 48 uses the generic kernels
    P2.close()


@pytest.mark.parametrize("kind,n", [("laplace", 10), ("helmholtz", 14), ("helmholtz", 20), ("maxwell", 22),
                                    ("helmholtz", 50)])
def test_radix_5_7_11_sizes(vie, kind, n):
    """Grid sizes with factors 5, 7, 11 (the paper's n = 50, 70, ..., 220 need them)."""
    import torch

    p = make_problem(kind, n, 2.0, False, seed=3)
    P = vie.Problem(kind, n, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
    op = operators.OracleProblem.from_problem(p)
    x = vi.random_field(n, op.ncomp, 12)[0]
    for prec, dt, tol in ((vie.VIE_FP64, torch.complex128, 1e-12), (vie.VIE_FP32, torch.complex64, 2e-5)):
        xd = to_dev(x, dt)
        yd = torch.empty_like(xd)
        P.apply(xd, yd, prec)
        torch.cuda.synchronize()
        ref = op.apply(x if prec == vie.VIE_FP64 else x.astype(np.complex64).astype(np.complex128))
        assert rel(yd.cpu().numpy(), ref) <= tol
    P.close()


@pytest.mark.parametrize("kind,n,mu", [("laplace", 5, False), ("helmholtz", 9, False), ("maxwell", 15, True),
                                       ("helmholtz", 21, False)])
def test_odd_grid_sizes(vie, kind, n, mu):
    """Odd n: the oversampled set-up grid 3n is odd (a symmetric frequency cut with no
    Nyquist entry), and the n^2 x-lines leave the last tile of the generic x passes
    partly empty.  FP64, double-word and FP32 applies and an FP64 solve against the oracle."""
    import torch

    p = make_problem(kind, n, 2.0, mu, seed=7)
    P = vie.Problem(kind, n, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
    try:
        op = operators.OracleProblem.from_problem(p)
        x = vi.random_field(n, op.ncomp, 13)[0]
        for prec, dt, tol in ((vie.VIE_FP64, torch.complex128, 1e-12), (vie.VIE_DF64, torch.complex128, 1e-12),
                              (vie.VIE_FP32, torch.complex64, 2e-5)):
            xd = to_dev(x, dt)
            yd = torch.empty_like(xd)
            P.apply(xd, yd, prec)
            torch.cuda.synchronize()
            ref = op.apply(x if dt == torch.complex128 else x.astype(np.complex64).astype(np.complex128))
            assert rel(yd.cpu().numpy(), ref) <= tol, prec
        d = p.directions[0]
        pol = p.polarisations[0] if kind == "maxwell" else None
        b = torch.empty((op.ncomp, n, n, n), dtype=torch.complex128, device="cuda:0")
        P.rhs(d, pol, 1, b)
        bo = op.rhs(d, pol)
        assert rel(b.cpu().numpy(), bo) <= 1e-12
        J = torch.zeros_like(b)
        st, info = P.solve(b, J, tol=1e-11, restart=60)
        Jo, _ = solvers.gmres(op.apply, bo, tol=1e-13, restart=60)
        assert info.rel_residual <= 1e-11
        assert rel(J.cpu().numpy(), Jo) <= 1e-9
    finally:
        P.close()


@pytest.mark.parametrize("medium,kind", [("eps234", "helmholtz"), ("eps_dense", "maxwell")])
def test_bicgstab_matches_oracle_on_paper_media(vie, medium, kind):
    """The paper's solver (Sec. 5) on its media (Sec. 5.2): same solution and matvec count as the oracle."""
    import torch

    n, size = 20, 1.0
    eps = vi.paper_medium(medium, n, 0.0, 1.0)
    omega = 2 * math.pi * size
    P = vie.Problem(kind, n, 0.0, 1.0, omega, to_dev(eps.reshape(9, -1)))
    op = operators.OracleProblem(kind, n, 0.0, 1.0, omega, eps)
    d = np.array([1.0, 0.0, 0.0])
    pol = np.array([0.0, 0.0, 1.0])
    b = torch.empty((3, n, n, n), dtype=torch.complex128, device="cuda:0")
    P.rhs(d, pol if kind == "maxwell" else None, 1, b)
    J = torch.zeros_like(b)
    st, info = P.solve(b, J, tol=1e-12, max_inner=500, mode=vie.VIE_SOLVE_BICGSTAB)
    Jo, io = solvers.bicgstab(op.apply, op.rhs(d, pol if kind == "maxwell" else None), tol=1e-12)
    assert io["converged"] and info.rel_residual <= 1e-12
    assert rel(J.cpu().numpy(), Jo) <= 1e-10
    assert abs(info.applies_fp64 - io["applies"]) <= 2
    P.close()
