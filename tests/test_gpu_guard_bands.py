"""Guard bands: every entry point writes its output buffer and nothing next to it.

Each vector handed to the library is a view into a larger buffer whose margins
hold a sentinel (exactly representable in FP32 and FP64).  After the call the
margins must be bit-identical and the input untouched: a pad, gather or
epilogue index that runs past the end of a line, a tile or the batch would
show up here even where the values inside the buffer are right.  Fast
(register-resident) and generic sizes, an odd size, Maxwell with mu, a batch
of two and all three precisions.
"""
import math

import numpy as np
import pytest

import vie_inputs as vi
from gpu_common import eps_dev, mu_dev, vie  # noqa: F401

pytestmark = pytest.mark.gpu

SENTINEL = complex(12345.25, -678.5)
GUARD = 4096  # elements on each side


def guarded(shape, dtype, fill=None):
    """(buffer, view): the view holds `fill` (or the sentinel), the margins the sentinel."""
    import torch

    size = math.prod(shape)
    buf = torch.full((GUARD + size + GUARD,), SENTINEL, dtype=dtype, device="cuda:0")
    view = buf[GUARD:GUARD + size].view(shape)
    if fill is not None:
        view.copy_(fill)
    return buf, view


def margins_intact(buf):
    import torch

    sent = torch.full((GUARD,), SENTINEL, dtype=buf.dtype, device=buf.device)
    return torch.equal(buf[:GUARD], sent) and torch.equal(buf[-GUARD:], sent)


CASES = [("helmholtz", 32, False, 1), ("helmholtz", 128, False, 1), ("maxwell", 16, True, 2), ("laplace", 9, False, 2)]


@pytest.mark.parametrize("kind,n,with_mu,nrhs", CASES, ids=lambda v: str(v))
def test_apply_rhs_and_scattered_field_stay_inside_their_buffers(vie, kind, n, with_mu, nrhs):
    import torch

    if kind == "laplace":
        p = vi.laplace_bump_problem(n=n, seed=5)
    elif kind == "helmholtz":
        p = vi.helmholtz_problem(n=n, wavelengths=3.0, seed=5)
    else:
        p = vi.maxwell_problem(n=n, wavelengths=2.0, with_mu=with_mu, seed=5)
    P = vie.Problem(kind, n, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
    try:
        c = P.ncomp
        shape = (nrhs, c, n, n, n)
        x64 = torch.from_numpy(vi.random_field(n, c, 8, nrhs=nrhs)).to("cuda:0")
        for prec, dt in ((vie.VIE_FP64, torch.complex128), (vie.VIE_DF64, torch.complex128),
                         (vie.VIE_FP32, torch.complex64)):
            xbuf, x = guarded(shape, dt, x64.to(dt))
            ybuf, y = guarded(shape, dt)
            x_before = x.clone()
            P.apply(x, y, prec, nrhs=nrhs)
            torch.cuda.synchronize()
            assert margins_intact(ybuf) and margins_intact(xbuf), prec
            assert torch.equal(x, x_before), prec
            assert bool(torch.isfinite(torch.view_as_real(y)).all()), prec
        dirs = np.tile(p.directions[:1], (nrhs, 1))
        pols = np.tile(p.polarisations[:1], (nrhs, 1)) if kind == "maxwell" else None
        bbuf, b = guarded(shape, torch.complex128)
        P.rhs(dirs, pols, nrhs, b)
        torch.cuda.synchronize()
        assert margins_intact(bbuf)
        cout = 6 if kind == "maxwell" else 1
        fbuf, f = guarded((nrhs, cout, n, n, n), torch.complex128)
        P.eval_scattered(x64, f, nrhs=nrhs)
        torch.cuda.synchronize()
        assert margins_intact(fbuf)
    finally:
        P.close()


@pytest.mark.parametrize("mode_name", ["fp64", "mixed"])
def test_solve_stays_inside_its_buffers(vie, mode_name):
    import torch

    n, nrhs = 24, 2
    p = vi.helmholtz_problem(n=n, wavelengths=3.0, seed=6)
    P = vie.Problem("helmholtz", n, p.lo, p.hi, p.omega, eps_dev(p))
    try:
        shape = (nrhs, 3, n, n, n)
        b = torch.empty(shape, dtype=torch.complex128, device="cuda:0")
        P.rhs(np.tile(p.directions[:1], (nrhs, 1)), None, nrhs, b)
        bbuf, bg = guarded(shape, torch.complex128, b)
        jbuf, J = guarded(shape, torch.complex128, torch.zeros(shape, dtype=torch.complex128, device="cuda:0"))
        mode = vie.VIE_SOLVE_FP64 if mode_name == "fp64" else vie.VIE_SOLVE_MIXED
        st, info = P.solve(bg, J, tol=1e-8, restart=30, mode=mode, nrhs=nrhs)
        torch.cuda.synchronize()
        assert info.rel_residual <= 1e-8
        assert margins_intact(jbuf) and margins_intact(bbuf)
        assert torch.equal(bg, b)
    finally:
        P.close()
