"""vie_apply_static: the operator apply for callers that cannot allocate.

Solvers inside frameworks that own all device memory through their own arena
or pool, and latency-bound loops that must not take the device-wide
synchronisation of cudaMalloc/cudaFree (or risk running out of memory in the
middle of a run), cannot let the library allocate its scratch when they apply
the operator.  vie_apply_static runs the same pipeline with its scratch in a
fixed 64 MiB device array.

The file name sorts last so that a run stopping at its first failure has run
every other test before this one.  Nothing here depends on that order: the
array is reserved when the library loads, and each test makes its own
schedule choice (vie_apply or vie_tune) before the static call.
"""
import numpy as np
import pytest

import vie_inputs as vi
from oracle import operators

from gpu_common import eps_dev, mu_dev, rel, to_dev, vie  # noqa: F401

pytestmark = pytest.mark.gpu

CASES = [
    # fast sizes (register-resident passes): 2n = 96, 64, 128
    ("helmholtz", 48, False, "fp32", 1),
    ("helmholtz", 48, False, "fp64", 1),
    ("maxwell", 32, True, "fp32", 1),
    ("laplace", 64, False, "fp32", 1),
    # generic Stockham sizes: 2n = 48 (radix 2/3) and odd n = 33 (2n = 66, radix 11)
    ("helmholtz", 24, False, "fp32", 1),
    ("helmholtz", 24, False, "fp64", 1),
    ("helmholtz", 33, False, "fp32", 1),
    # two right-hand sides in one call (workspace of nrhs = 2 within the 64 MiB)
    ("helmholtz", 32, False, "fp32", 2),
    ("maxwell", 24, True, "fp64", 2),
]


def _problem(kind, n, with_mu):
    if kind == "laplace":
        return vi.laplace_bump_problem(n=n, seed=2)
    if kind == "helmholtz":
        return vi.helmholtz_problem(n=n, wavelengths=3.0, seed=2)
    return vi.maxwell_problem(n=n, wavelengths=2.0, with_mu=with_mu, seed=2)


@pytest.mark.parametrize("kind,n,with_mu,prec_name,nrhs", CASES)
def test_static_apply_equals_apply_twice(vie, kind, n, with_mu, prec_name, nrhs):
    """Two calls in a row through the C ABI give vie_apply's result bit for bit
    (same kernels, same schedule, scratch in the static array); the result also
    matches the FP64 oracle within the parity tolerance of its precision."""
    import torch

    prec = vie.VIE_FP32 if prec_name == "fp32" else vie.VIE_FP64
    dt = torch.complex64 if prec_name == "fp32" else torch.complex128
    tol = 2e-5 if prec_name == "fp32" else 1e-12
    p = _problem(kind, n, with_mu)
    P = vie.Problem(kind, n, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
    xh = vi.random_field(n, P.ncomp, 21, nrhs=nrhs)
    if nrhs == 1:
        xh = xh[0]
    x = to_dev(xh, dt)
    y_ref = torch.empty_like(x)
    P.apply(x, y_ref, prec, nrhs=nrhs)  # ordinary entry point: allocates its workspace, picks the schedule
    torch.cuda.synchronize()
    for call in range(2):  # two calls in a row share (and reuse) the static scratch
        y = torch.full_like(x, float("nan"))
        vie.vie_apply_static(P.handle, x, y, prec, nrhs)
        torch.cuda.synchronize()
        assert torch.equal(y, y_ref), (call, kind, n, prec_name, nrhs)
    op = operators.OracleProblem.from_problem(p)
    xs = xh if nrhs > 1 else xh[None]
    ys = y_ref.cpu().numpy().reshape(xs.shape)
    for r in range(nrhs):
        x64 = xs[r].astype(np.complex64).astype(np.complex128) if prec_name == "fp32" else xs[r]
        assert rel(ys[r], op.apply(x64)) <= tol, (r, kind, n, prec_name)
    P.close()


def test_static_apply_allocates_nothing(vie):
    """Ten calls after the first leave the device's free memory unchanged (no
    allocation, also none that a memory pool would keep)."""
    import torch

    n = 32
    p = _problem("helmholtz", n, False)
    P = vie.Problem("helmholtz", n, p.lo, p.hi, p.omega, eps_dev(p))
    x = to_dev(vi.random_field(n, 3, 5)[0], torch.complex64)
    y = torch.empty_like(x)
    P.tune(vie.VIE_FP32)
    vie.vie_apply_static(P.handle, x, y, vie.VIE_FP32)  # first call: looks up the array's address
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(10):
        vie.vie_apply_static(P.handle, x, y, vie.VIE_FP32)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    P.close()


def test_static_apply_rejects_oversize_and_unchosen_schedule(vie):
    import torch

    p = vi.helmholtz_problem(n=96, wavelengths=2.0, seed=1)
    P = vie.Problem("helmholtz", 96, p.lo, p.hi, p.omega, eps_dev(p))
    x = torch.zeros((3, 96, 96, 96), dtype=torch.complex64, device="cuda:0")
    y = torch.empty_like(x)
    P.apply(x, y, vie.VIE_FP32)
    with pytest.raises(vie.VieError) as ei:  # 96^3 needs 127 MB of scratch > 64 MiB
        vie.vie_apply_static(P.handle, x, y, vie.VIE_FP32)
    assert ei.value.status == vie.VIE_EINVAL
    P.close()
    # Laplace n = 32 in FP64: unless an earlier test of this process chose that
    # shape's schedule (the choice is process-wide, keyed by n, precision and kind),
    # the static call is refused until one is chosen
    q = vi.laplace_bump_problem(n=32, seed=1)
    Q = vie.Problem("laplace", 32, q.lo, q.hi, 0.0, eps_dev(q))
    x = torch.zeros((3, 32, 32, 32), dtype=torch.complex128, device="cuda:0")
    _static_served_or_refused(vie, Q, x)
    Q.tune(vie.VIE_FP64)
    vie.vie_apply_static(Q.handle, x, torch.empty_like(x), vie.VIE_FP64)
    # a second handle of the same shape reuses the process-wide choice: no refusal
    R = vie.Problem("laplace", 32, q.lo, q.hi, 0.0, eps_dev(q))
    vie.vie_apply_static(R.handle, x, torch.empty_like(x), vie.VIE_FP64)
    N = 32 ** 3
    buf = torch.zeros(3 * N + 1, dtype=torch.complex128, device="cuda:0")
    with pytest.raises(vie.VieError) as ei:  # x and y one element apart share all but one element
        vie.vie_apply_static(Q.handle, buf[1:].view(3, 32, 32, 32), buf[:3 * N].view(3, 32, 32, 32), vie.VIE_FP64)
    assert ei.value.status == vie.VIE_EINVAL
    with pytest.raises(vie.VieError) as ei:  # double-word arithmetic is not offered here
        vie.vie_apply_static(Q.handle, x, torch.empty_like(x), vie.VIE_DF64)
    assert ei.value.status == vie.VIE_EINVAL
    R.close()
    Q.close()


def _static_served_or_refused(vie, Q, x):
    """The static call either runs (the shape's schedule is already known to the
    process) or is refused with VIE_EINVAL; nothing else."""
    import torch

    try:
        vie.vie_apply_static(Q.handle, x, torch.empty_like(x), vie.VIE_FP64)
    except vie.VieError as e:
        assert e.status == vie.VIE_EINVAL
