"""The Python binding refuses tensors the library would access out of bounds (no GPU).

The C ABI takes raw device pointers and trusts the sizes it is given; the
binding, which sees the tensors, refuses (VIE_EINVAL, before the library is
called) a host tensor, a strided view, or a buffer smaller than the bytes the
call's grid size, component count, batch size and precision imply.
"""
import ctypes

import pytest

import paper_1805_04791_gb300 as vie


class FakeCudaTensor:
    """Stands in for a CUDA tensor: only what the binding's checks look at."""

    def __init__(self, numel, elem, contiguous=True):
        self._n, self._e, self._c = numel, elem, contiguous
        self.is_cuda = True
        self.device = "cuda:0"

    def numel(self):
        return self._n

    def element_size(self):
        return self._e

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        return 0x10000


@pytest.fixture(autouse=True)
def no_library(monkeypatch):
    """Every call here must be refused before the library is reached."""

    def reached(*a, **k):
        raise AssertionError("the library was called with an unchecked buffer")

    monkeypatch.setattr(vie, "load", reached)


@pytest.fixture
def handle():
    h = ctypes.c_void_p(0xABC0)
    vie._SHAPES[h.value] = (8, 3, vie.VIE_LAPLACE)  # n = 8, 3 components
    yield h
    vie._SHAPES.pop(h.value, None)


def status_of(call):
    with pytest.raises(vie.VieError) as ei:
        call()
    return ei.value.status


def test_host_and_strided_tensors_are_refused():
    torch = pytest.importorskip("torch")
    assert status_of(lambda: vie._dev(torch.zeros(8, dtype=torch.complex128), 16, "x")) == vie.VIE_EINVAL
    assert status_of(lambda: vie._dev(FakeCudaTensor(100, 16, contiguous=False), 16, "x")) == vie.VIE_EINVAL
    assert status_of(lambda: vie._dev(None, 16, "x")) == vie.VIE_EINVAL
    assert vie._dev(FakeCudaTensor(1, 16), 16, "x").value == 0x10000


def test_sizes_follow_grid_components_batch_and_precision(handle):
    N = 8 ** 3
    assert vie._vec_bytes(handle, None, 1, 16) == 16 * 3 * N
    assert vie._vec_bytes(handle, None, 4, 8) == 8 * 4 * 3 * N
    assert vie._vec_bytes(handle, lambda sh: 1, 2, 16) == 16 * 2 * N
    assert vie._vec_bytes(ctypes.c_void_p(0x1230), None, 1, 16) is None  # unknown handle: size unchecked


def test_calls_refuse_short_buffers_before_the_library(handle):
    N = 8 ** 3
    ok64, ok32 = FakeCudaTensor(3 * N, 16), FakeCudaTensor(3 * N, 8)
    short64 = FakeCudaTensor(3 * N - 1, 16)
    # FP64 apply needs 16 bytes per value: an FP32-sized buffer is half too small
    assert status_of(lambda: vie.vie_apply(handle, ok32, ok64, vie.VIE_FP64)) == vie.VIE_EINVAL
    assert status_of(lambda: vie.vie_apply(handle, ok64, short64, vie.VIE_DF64)) == vie.VIE_EINVAL
    assert status_of(lambda: vie.vie_apply(handle, ok64, ok64, vie.VIE_FP64, nrhs=2)) == vie.VIE_EINVAL
    assert status_of(lambda: vie.vie_apply_static(handle, ok32, FakeCudaTensor(3 * N - 1, 8), vie.VIE_FP32)) \
        == vie.VIE_EINVAL
    opts = vie.SolveOpts(1e-8, 20, 5, 100, 1e-5, vie.VIE_SOLVE_MIXED, 2)
    assert status_of(lambda: vie.vie_solve(handle, ok64, ok64, opts)) == vie.VIE_EINVAL
    assert status_of(lambda: vie.vie_rhs_plane_wave(handle, [0, 0, 1], None, 1, short64)) == vie.VIE_EINVAL
    assert status_of(lambda: vie.vie_rhs_plane_wave(handle, [0, 0, 1], None, 2, FakeCudaTensor(6 * N, 16))) \
        == vie.VIE_EINVAL  # d holds one direction for two right-hand sides
    # the scattered potential has one component: J needs 3 N values, the output N
    assert status_of(lambda: vie.vie_eval_scattered(handle, short64, FakeCudaTensor(N, 16))) == vie.VIE_EINVAL
    assert status_of(lambda: vie.vie_eval_scattered(handle, ok64, FakeCudaTensor(N - 1, 16))) == vie.VIE_EINVAL


def test_create_refuses_a_medium_smaller_than_the_grid():
    eps8 = FakeCudaTensor(9 * 8 ** 3, 16)
    assert status_of(lambda: vie.vie_problem_create(vie.VIE_LAPLACE, 10, -1.0, 1.0, 0.0, eps8)) == vie.VIE_EINVAL
    assert status_of(lambda: vie.vie_problem_create(vie.VIE_MAXWELL, 8, -1.0, 1.0, 1.0, eps8,
                                                    FakeCudaTensor(9 * 8 ** 3 - 1, 16))) == vie.VIE_EINVAL
