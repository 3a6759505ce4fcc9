"""Shared helpers of the GPU parity tests (the oracle is the checker)."""
import numpy as np
import pytest

import vie_inputs as vi


@pytest.fixture(scope="session")
def vie():
    import torch

    import __graft_entry__ as entry

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    entry.build()
    import paper_1805_04791_gb300 as mod

    mod.load()
    return mod


def to_dev(a, dtype=None):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to("cuda:0")


def eps_dev(p):
    return to_dev(p.eps.reshape(9, -1))


def mu_dev(p):
    return None if p.mu is None else to_dev(p.mu.reshape(9, -1))


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
