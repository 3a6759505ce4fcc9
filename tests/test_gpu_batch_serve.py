"""GPU: batched right-hand sides and the serving loop (through the C ABI)."""
import numpy as np
import pytest

import vie_inputs as vi
from oracle import operators, solvers

from gpu_common import eps_dev, mu_dev, rel, to_dev, vie  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("group_max", ["1", "2", "64"])
def test_batched_mixed_solve_matches_oracle(vie, monkeypatch, group_max):
    """Maxwell with mu, 4 right-hand sides (2 directions x 2 polarisations) solved in
    lockstep groups (group size forced through VIE_GROUP_MAX); each equals the oracle."""
    import torch

    monkeypatch.setenv("VIE_GROUP_MAX", group_max)
    n = 12
    p = vi.maxwell_problem(n=n, wavelengths=2.0, ndirs=2, npol=2, with_mu=True, seed=5)
    P = vie.Problem("maxwell", n, p.lo, p.hi, p.omega, eps_dev(p), mu_dev(p))
    op = operators.OracleProblem.from_problem(p)
    nr = p.nrhs
    b = torch.empty((nr, 6, n, n, n), dtype=torch.complex128, device="cuda:0")
    P.rhs(p.directions, p.polarisations, nr, b)
    J = torch.zeros_like(b)
    st, info = P.solve(b, J, tol=1e-10, restart=30, mode=vie.VIE_SOLVE_MIXED, nrhs=nr)
    assert info.rel_residual <= 1e-10
    for r in range(nr):
        Jo, _ = solvers.gmres(op.apply, op.rhs(p.directions[r], p.polarisations[r]), tol=1e-13, restart=60)
        assert rel(J[r].cpu().numpy(), Jo) <= 1e-8
    P.close()


def test_batched_equals_single_fp64(vie, monkeypatch):
    """A lockstep group returns the same solutions as one-at-a-time solves."""
    import torch

    n = 16
    p = vi.helmholtz_problem(n=n, wavelengths=3.0, nrhs=3, seed=9)
    P = vie.Problem("helmholtz", n, p.lo, p.hi, p.omega, eps_dev(p))
    b = torch.empty((3, 3, n, n, n), dtype=torch.complex128, device="cuda:0")
    P.rhs(p.directions, None, 3, b)
    Jb = torch.zeros_like(b)
    P.solve(b, Jb, tol=1e-11, restart=40, mode=vie.VIE_SOLVE_FP64, nrhs=3)
    monkeypatch.setenv("VIE_GROUP_MAX", "1")
    Js = torch.zeros_like(b)
    P.solve(b, Js, tol=1e-11, restart=40, mode=vie.VIE_SOLVE_FP64, nrhs=3)
    assert rel(Jb.cpu().numpy(), Js.cpu().numpy()) <= 1e-10
    P.close()


def _serving_oracle_solution(req):
    """The oracle's FP64 GMRES solution of one served request: the same medium
    formula (the anisotropic bump with the request's seed, evaluated on the
    host), frequency, incident wave and discrete operator."""
    rng = vi.SplitMix64(req.seed)
    eps = vi.anisotropic_bump(req.n, -1.0, 1.0, 0.5, 0.1, rng).real.astype(np.complex128)
    omega = 2.0 * np.pi * req.wavelengths / 2.0
    op = operators.OracleProblem(req.kind, req.n, -1.0, 1.0, omega, eps, None)
    pol = req.polarisation if req.kind == "maxwell" else None
    Jo, info = solvers.gmres(op.apply, op.rhs(req.direction, pol), tol=1e-12, restart=60, maxiter=800)
    assert info["converged"]
    return Jo


def test_serving_mix_completes_and_is_mix_invariant(vie):
    """Requests of different sizes and kinds overlap on the device; a request's
    result is the same alone and inside the mix, and every served solution
    equals the oracle's solution of that request."""
    from paper_1805_04791_gb300 import serve

    reqs = vi.serving_mix(10, rate_per_s=200.0, seed=4, sizes=(16, 24, 32), wl_range=(1.0, 3.0))
    target = reqs[3]
    alone = serve.Server(budget_bytes=8e9, max_slots=1, keep_solutions=True, tol=1e-10).run([target])
    assert alone.results[0].status == "ok", alone.results[0].status
    mix = serve.Server(budget_bytes=8e9, max_slots=6, keep_solutions=True, tol=1e-10).run(reqs)
    s = mix.summary()
    assert s["completed"] == 10, [r.status for r in mix.results]
    assert s["peak_inflight"] >= 2  # requests really overlapped
    by_id = {r.rid: r for r in reqs}
    for r in mix.results:
        assert r.rel_residual <= 1e-10
        # mixed solve to 1e-10 on a second-kind operator: solution error ~1e-9
        assert rel(r.solution, _serving_oracle_solution(by_id[r.rid])) <= 1e-8, (r.rid, r.kind, r.n)
    got = [r for r in mix.results if r.rid == target.rid][0]
    a, m = alone.results[0].solution, got.solution
    assert rel(m, a) <= 1e-12
