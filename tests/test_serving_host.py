"""Host-side tests of the serving loop and the device medium generator (no GPU).

The admission logic is exercised with a fake solver that sleeps instead of
launching kernels: the HBM budget and the slot limit must never be exceeded,
waiting requests are admitted shortest first unless one has waited past the
aging limit (then oldest first), and every request completes.
"""
import threading
import time

import numpy as np
import pytest

import vie_inputs as vi


def test_serving_mix_is_seeded_and_poisson():
    a = vi.serving_mix(200, rate_per_s=50.0, seed=3)
    b = vi.serving_mix(200, rate_per_s=50.0, seed=3)
    assert [r.arrival_s for r in a] == [r.arrival_s for r in b]
    assert [(r.kind, r.n, r.seed) for r in a] == [(r.kind, r.n, r.seed) for r in b]
    gaps = np.diff([0.0] + [r.arrival_s for r in a])
    assert abs(gaps.mean() - 1 / 50.0) < 0.25 / 50.0  # exponential inter-arrivals, mean 1/rate
    assert set(r.n for r in a) <= {32, 48, 64, 96, 128, 192}
    assert {r.kind for r in a} == {"helmholtz", "maxwell"}
    for r in a:
        assert 1.0 <= r.wavelengths <= 8.0
        assert abs(np.linalg.norm(r.direction) - 1) < 1e-12 and abs(r.direction @ r.polarisation) < 1e-12


def test_torch_medium_matches_numpy_generator():
    torch = pytest.importorskip("torch")
    n, seed = 10, 77
    e_t = vi.bump_medium_torch(n, seed, torch.device("cpu")).numpy()
    rng = vi.SplitMix64(seed)
    e_n = vi.anisotropic_bump(n, -1.0, 1.0, 0.5, 0.1, rng).reshape(9, -1)
    assert np.max(np.abs(e_t - e_n)) <= 1e-15


class FakeServer:
    """Server with the solve replaced by a sleep; checks the admission invariants."""

    def __init__(self, budget, slots):
        from paper_1805_04791_gb300 import serve

        self.mod = serve
        self.budget = budget
        self.slots = slots
        self.lock = threading.Lock()
        self.used = 0
        self.inflight = 0
        self.violations = []
        self.order = []
        self.kw = {}

    def make(self):
        outer = self

        class S(self.mod.Server):
            def request_bytes(self, req):
                return req.n * 1000

            def _solve(self, req, res, done_cb):
                with outer.lock:
                    outer.used += req.n * 1000
                    outer.inflight += 1
                    outer.order.append(req.rid)
                    if outer.used > outer.budget or outer.inflight > outer.slots:
                        outer.violations.append((req.rid, outer.used, outer.inflight))
                time.sleep(0.002 * req.n / 32)
                res.status = "ok"
                res.rel_residual = 0.0
                with outer.lock:
                    outer.used -= req.n * 1000
                    outer.inflight -= 1
                done_cb(res)

        return S(budget_bytes=self.budget, max_slots=self.slots, **self.kw)


def test_admission_respects_budget_and_slots():
    pytest.importorskip("torch")
    reqs = vi.serving_mix(60, rate_per_s=2000.0, seed=1)
    fake = FakeServer(budget=300_000, slots=4)
    stats = fake.make().run(reqs)
    assert not fake.violations
    s = stats.summary()
    assert s["completed"] == 60 and s["failed"] == 0
    assert stats.peak_bytes <= 300_000 and stats.peak_slots <= 4
    assert all(r.done_s >= r.admit_s >= r.arrival_s - 1e-9 for r in stats.results)


def test_oversized_request_is_rejected_not_hung():
    pytest.importorskip("torch")
    reqs = vi.serving_mix(10, rate_per_s=1000.0, seed=2)
    fake = FakeServer(budget=100_000, slots=8)  # n >= 128 needs > budget
    stats = fake.make().run(reqs)
    for r in stats.results:
        big = r.n * 1000 > 100_000
        assert (r.status.startswith("rejected")) == big


def test_failed_request_releases_its_problem(monkeypatch):
    """A request whose solve raises is reported as an error, its problem handle is
    closed (its device memory returns before its slot does) and the slot is freed."""
    torch = pytest.importorskip("torch")
    import contextlib

    from paper_1805_04791_gb300 import serve

    closed = []

    class FakeProblem:
        def __init__(self, kind, n, lo, hi, omega, eps, mu=None, stream=None):
            self.ncomp = 3

        def rhs(self, *a, **k):
            pass

        def solve(self, *a, **k):
            raise RuntimeError("solver failed")

        def close(self):
            closed.append(True)

    class FakeStream:
        def synchronize(self):
            pass

    monkeypatch.setattr(serve, "Problem", FakeProblem)
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(vi, "bump_medium_torch", lambda n, seed, dev: torch.zeros(9, n ** 3, dtype=torch.complex128))
    real_empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, **k: real_empty(*a, **{**k, "device": "cpu"}))
    req = vi.serving_mix(1, rate_per_s=10.0, seed=4)[0]
    res = serve.ServeResult(req.rid, req.kind, 8, 0.0)
    req.n = 8
    done = []
    serve.Server()._solve(req, res, done.append)
    assert res.status == "error: solver failed"
    assert closed == [True] and done == [res]


def _burst(sizes, t=0.0):
    """Requests of the given grid sizes, all arriving at time t."""
    base = vi.serving_mix(len(sizes), rate_per_s=100.0, seed=9)
    for i, (r, n) in enumerate(zip(base, sizes)):
        r.rid, r.n, r.arrival_s = i, n, t
    return base


def test_shortest_job_first_admission():
    """One slot, a simultaneous burst: after the first admission the waiting
    requests are admitted in increasing grid size."""
    pytest.importorskip("torch")
    sizes = [192, 32, 128, 48, 96, 64, 32, 192]
    fake = FakeServer(budget=10 ** 9, slots=1)
    fake.kw = {"max_wait_s": 60.0}
    fake.make().run(_burst(sizes))
    ns = [sizes[rid] for rid in fake.order]
    assert ns == sorted(ns), ns


def test_aged_requests_go_first():
    """With an aging limit of zero every waiting request counts as aged, and
    admission falls back to arrival order (the FIFO policy gives the same)."""
    pytest.importorskip("torch")
    sizes = [192, 32, 128, 48, 96]
    reqs = _burst(sizes)
    for i, r in enumerate(reqs):
        r.arrival_s = 0.001 * i
    for kw in ({"max_wait_s": 0.0}, {"policy": "fifo"}):
        fake = FakeServer(budget=10 ** 9, slots=1)
        fake.kw = kw
        fake.make().run(reqs)
        assert fake.order == list(range(len(sizes))), (kw, fake.order)
