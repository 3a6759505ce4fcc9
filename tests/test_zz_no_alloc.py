"""vie_apply_static: the operator apply for callers that cannot allocate.

Code recorded into a CUDA graph by stream capture, solvers inside frameworks
that own all device memory through their own arena, and latency-bound loops
that must not take the device-wide synchronisation of cudaMalloc/cudaFree
cannot let the library allocate its scratch when they apply the operator.
vie_apply_static runs the same pipeline with its scratch in a fixed 64 MiB
device array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import vie_inputs as vi

from gpu_common import eps_dev, mu_dev, rel, to_dev, vie  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,n,with_mu,prec_name", [("helmholtz", 48, False, "fp32"), ("helmholtz", 48, False, "fp64"),
                                                      ("maxwell", 32, True, "fp32"), ("laplace", 64, False, "fp32")])
def test_static_apply_matches_apply_twice(vie, kind, n, with_mu, prec_name):
    import torch

    prec = vie.VIE_FP32 if prec_name == "fp32" else vie.VIE_FP64
    dt = torch.complex64 if prec_name == "fp32" else torch.complex128
    tol = 2e-5 if prec_name == "fp32" else 1e-12
    if kind == "laplace":
        p = vi.laplace_bump_problem(n=n, seed=2)
    elif kind == "helmholtz":
        p = vi.helmholtz_problem(n=n, wavelengths=3.0, seed=2)
    else:
        p = vi.maxwell_problem(n=n, wavelengths=2.0, with_mu=with_mu, seed=2)
    P = vie.Problem(kind, n, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
    x = to_dev(vi.random_field(n, P.ncomp, 21)[0], dt)
    y_ref = torch.empty_like(x)
    P.apply(x, y_ref, prec)  # ordinary entry point: allocates its workspace, picks the z-pass schedule
    torch.cuda.synchronize()
    ref = y_ref.cpu().numpy()
    for call in range(2):  # two calls in a row share (and reuse) the static scratch
        y = torch.full_like(x, float("nan"))
        vie.vie_apply_static(P.handle, x, y, prec)
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), ref) <= tol, (call, kind, n, prec_name)
    P.close()


def test_static_apply_rejects_oversize_and_untuned(vie):
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
    q = vi.helmholtz_problem(n=32, wavelengths=2.0, seed=1)
    Q = vie.Problem("helmholtz", 32, q.lo, q.hi, q.omega, eps_dev(q))
    x = torch.zeros((3, 32, 32, 32), dtype=torch.complex128, device="cuda:0")
    with pytest.raises(vie.VieError) as ei:  # schedule for FP64 not chosen yet
        vie.vie_apply_static(Q.handle, x, torch.empty_like(x), vie.VIE_FP64)
    assert ei.value.status == vie.VIE_EINVAL
    Q.tune(vie.VIE_FP64)
    vie.vie_apply_static(Q.handle, x, torch.empty_like(x), vie.VIE_FP64)
    N = 32 ** 3
    buf = torch.zeros(3 * N + 1, dtype=torch.complex128, device="cuda:0")
    with pytest.raises(vie.VieError) as ei:  # x and y one element apart share all but one element
        vie.vie_apply_static(Q.handle, buf[1:].view(3, 32, 32, 32), buf[:3 * N].view(3, 32, 32, 32), vie.VIE_FP64)
    assert ei.value.status == vie.VIE_EINVAL
    Q.close()
