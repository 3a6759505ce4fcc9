"""Failure statuses, injected on the host (no GPU fault, trap or hang).

* A NaN in the right-hand side returns VIE_ENAN before any iteration.
* A NaN in the initial guess makes the first residual non-finite: VIE_ENAN.
* An iteration limit below what the tolerance needs returns VIE_ENOCONV with the
  last iterate in J and its true residual in the info.
* After each failure the handle is still usable: a clean solve succeeds.
"""
import numpy as np
import pytest

import vie_inputs as vi
from gpu_common import eps_dev, vie  # noqa: F401

pytestmark = pytest.mark.gpu

MODES = ["fp64", "mixed", "bicgstab"]


def mode_of(vie, name):
    return {"fp64": vie.VIE_SOLVE_FP64, "mixed": vie.VIE_SOLVE_MIXED, "bicgstab": vie.VIE_SOLVE_BICGSTAB}[name]


def problem(vie, n=12):
    import torch

    p = vi.helmholtz_problem(n=n, wavelengths=2.0, seed=9)
    P = vie.Problem("helmholtz", n, p.lo, p.hi, p.omega, eps_dev(p))
    b = torch.empty((3, n, n, n), dtype=torch.complex128, device="cuda:0")
    P.rhs(p.directions[0], None, 1, b)
    return P, b


def clean_solve_works(vie, P, b, mode):
    import torch

    J = torch.zeros_like(b)
    st, info = P.solve(b, J, tol=1e-8, restart=30, mode=mode)
    return st == vie.VIE_OK and info.rel_residual <= 1e-8 and bool(torch.isfinite(torch.view_as_real(J)).all())


@pytest.mark.parametrize("mode_name", MODES)
def test_nan_right_hand_side_returns_enan(vie, mode_name):
    import torch

    P, b = problem(vie)
    try:
        m = mode_of(vie, mode_name)
        bad = b.clone()
        bad[1, 3, 4, 5] = complex(float("nan"), 0.0)
        J = torch.zeros_like(b)
        with pytest.raises(vie.VieError) as ei:
            P.solve(bad, J, tol=1e-8, restart=30, mode=m)
        assert ei.value.status == vie.VIE_ENAN
        assert clean_solve_works(vie, P, b, m)
    finally:
        P.close()


@pytest.mark.parametrize("mode_name", MODES)
def test_nan_initial_guess_returns_enan(vie, mode_name):
    import torch

    P, b = problem(vie)
    try:
        m = mode_of(vie, mode_name)
        J = torch.zeros_like(b)
        J[2, 1, 2, 3] = complex(float("nan"), 0.0)
        with pytest.raises(vie.VieError) as ei:
            P.solve(b, J, tol=1e-8, restart=30, mode=m)
        assert ei.value.status == vie.VIE_ENAN
        assert clean_solve_works(vie, P, b, m)
    finally:
        P.close()


@pytest.mark.parametrize("mode_name", MODES)
def test_iteration_limit_returns_enoconv_with_the_last_iterate(vie, mode_name):
    import torch

    P, b = problem(vie)
    try:
        m = mode_of(vie, mode_name)
        J = torch.zeros_like(b)
        st, info = P.solve(b, J, tol=1e-13, restart=5, max_outer=2, max_inner=3, mode=m, allow_noconv=True)
        assert st == vie.VIE_ENOCONV
        assert np.isfinite(info.rel_residual) and 1e-13 < info.rel_residual < 1.0
        assert bool(torch.isfinite(torch.view_as_real(J)).all()) and float(torch.linalg.vector_norm(J)) > 0.0
        with pytest.raises(vie.VieError) as ei:  # without allow_noconv the binding raises
            P.solve(b, torch.zeros_like(b), tol=1e-13, restart=5, max_outer=2, max_inner=3, mode=m)
        assert ei.value.status == vie.VIE_ENOCONV
        assert clean_solve_works(vie, P, b, m)
    finally:
        P.close()
