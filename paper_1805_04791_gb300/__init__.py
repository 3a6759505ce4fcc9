"""GB300 (sm_103a) FFT-accelerated volume-integral-equation solver.

Thin ctypes binding over the C ABI of ``include/vie.h`` (argument marshalling
only: every step of the computation runs in the library's CUDA kernels).
Functions carry the C names; ``Problem`` is a small convenience wrapper.
PyTorch provides device memory and streams: tensors are passed by
``data_ptr()`` and the stream by ``torch.cuda.current_stream().cuda_stream``.
Each tensor is checked before the call (a contiguous CUDA tensor with at least
the bytes the call's sizes imply), so a short, strided or host buffer is refused
with VIE_EINVAL instead of being accessed out of bounds by the kernels.

There is no CPU fallback: if the shared library is missing or fails to load,
importing the binding raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libvie_gb300.so")

VIE_OK, VIE_EINVAL, VIE_ENOMEM, VIE_ECUDA, VIE_ENOCONV, VIE_ENAN, VIE_ETIMEOUT, VIE_EBUSY = range(8)
VIE_LAPLACE, VIE_HELMHOLTZ, VIE_MAXWELL = range(3)
VIE_FP64, VIE_FP32, VIE_DF64 = 0, 1, 2  # VIE_DF64: FP64 vectors, double-word arithmetic
VIE_SOLVE_FP64, VIE_SOLVE_MIXED, VIE_SOLVE_BICGSTAB = 0, 1, 2
P3_VARIANTS = 19  # z-pass schedules vie_tune chooses from (include/vie.h)
KINDS = {"laplace": VIE_LAPLACE, "helmholtz": VIE_HELMHOLTZ, "maxwell": VIE_MAXWELL}
STATUS_NAMES = {0: "VIE_OK", 1: "VIE_EINVAL", 2: "VIE_ENOMEM", 3: "VIE_ECUDA", 4: "VIE_ENOCONV",
                5: "VIE_ENAN", 6: "VIE_ETIMEOUT", 7: "VIE_EBUSY"}

EXPORTED = ("vie_problem_create", "vie_problem_ncomp", "vie_apply", "vie_rhs_plane_wave", "vie_solve",
            "vie_eval_scattered", "vie_problem_bytes", "vie_problem_destroy", "vie_last_error",
            "vie_profile_begin", "vie_profile_end", "vie_tune", "vie_apply_static")


class VieError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_outer", ctypes.c_int),
                ("max_inner", ctypes.c_int), ("inner_tol", ctypes.c_double), ("mode", ctypes.c_int),
                ("nrhs", ctypes.c_int), ("check_fp64", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int), ("applies_fp32", ctypes.c_int),
                ("applies_fp64", ctypes.c_int), ("rel_residual", ctypes.c_double), ("t_solve", ctypes.c_double),
                ("t_precompute", ctypes.c_double), ("rel_residual_fp64", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, c_int, c_double = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.vie_problem_create.argtypes = [c_int, c_int, c_double, c_double, c_double, vp, vp, vp,
                                       ctypes.POINTER(vp)]
    lib.vie_problem_create.restype = c_int
    lib.vie_problem_ncomp.argtypes = [vp]
    lib.vie_problem_ncomp.restype = c_int
    lib.vie_apply.argtypes = [vp, vp, vp, c_int, c_int, vp]
    lib.vie_apply.restype = c_int
    lib.vie_rhs_plane_wave.argtypes = [vp, ctypes.POINTER(c_double), ctypes.POINTER(c_double), c_int, vp, vp]
    lib.vie_rhs_plane_wave.restype = c_int
    lib.vie_solve.argtypes = [vp, vp, vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp]
    lib.vie_solve.restype = c_int
    lib.vie_eval_scattered.argtypes = [vp, vp, vp, c_int, vp]
    lib.vie_eval_scattered.restype = c_int
    lib.vie_problem_bytes.argtypes = [c_int, c_int, c_int, c_int, c_int]
    lib.vie_problem_bytes.restype = ctypes.c_size_t
    lib.vie_problem_destroy.argtypes = [vp]
    lib.vie_problem_destroy.restype = c_int
    lib.vie_profile_begin.argtypes = [vp, c_int]
    lib.vie_profile_begin.restype = c_int
    lib.vie_profile_end.argtypes = [vp, ctypes.POINTER(c_double), c_int, ctypes.POINTER(c_int)]
    lib.vie_profile_end.restype = c_int
    lib.vie_apply_static.argtypes = [vp, vp, vp, c_int, c_int, vp]
    lib.vie_apply_static.restype = c_int
    lib.vie_tune.argtypes = [vp, c_int, ctypes.POINTER(c_int), vp]
    lib.vie_tune.restype = c_int
    lib.vie_last_error.argtypes = []
    lib.vie_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int, allow=(VIE_OK,)):
    if status not in allow:
        raise VieError(status, load().vie_last_error().decode())
    return status


def _stream(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# (n, components, kind) of every handle created through this binding: lets the
# calls below check that each tensor they hand to the library is big enough.
_SHAPES = {}


def _key(P):
    return P.value if isinstance(P, ctypes.c_void_p) else P


def _dev(t, need_bytes, what):
    """Device pointer of ``t``, refused (VIE_EINVAL, nothing launched) unless ``t`` is a
    contiguous CUDA tensor holding at least ``need_bytes`` bytes (None: size unknown).
    The library reads and writes exactly the bytes the call's sizes imply, so a
    smaller, strided or host buffer would be accessed out of bounds."""
    if t is None or not hasattr(t, "data_ptr"):
        raise VieError(VIE_EINVAL, f"{what}: expected a CUDA tensor")
    if not t.is_cuda:
        raise VieError(VIE_EINVAL, f"{what}: expected a CUDA tensor, got one on {t.device}")
    if not t.is_contiguous():
        raise VieError(VIE_EINVAL, f"{what}: expected a contiguous tensor")
    have = t.numel() * t.element_size()
    if need_bytes is not None and have < need_bytes:
        raise VieError(VIE_EINVAL, f"{what}: holds {have} bytes, the call accesses {need_bytes}")
    return ctypes.c_void_p(t.data_ptr())


def _vec_bytes(P, comps, nrhs, elem):
    """Bytes of nrhs fields of ``comps`` components on P's grid (None if P is unknown)."""
    sh = _SHAPES.get(_key(P))
    if sh is None:
        return None
    c = sh[1] if comps is None else comps(sh)
    return elem * max(nrhs, 0) * c * sh[0] ** 3


def _elem(precision):
    return 8 if precision == VIE_FP32 else 16


def _dvec(values):
    import numpy as np

    a = np.ascontiguousarray(np.asarray(values, dtype=np.float64).ravel())
    return (ctypes.c_double * a.size)(*a.tolist())


# ------------------------------------------------------------ C-named calls


def vie_problem_create(kind: int, n: int, lo: float, hi: float, omega: float, eps, mu=None, stream=None):
    need = 16 * 9 * max(n, 0) ** 3
    pe = _dev(eps, need, "eps")
    pm = None if mu is None else _dev(mu, need, "mu")
    h = ctypes.c_void_p()
    _check(load().vie_problem_create(kind, n, lo, hi, omega, pe, pm, _stream(stream), ctypes.byref(h)))
    _SHAPES[h.value] = (n, load().vie_problem_ncomp(h), kind)
    return h


def vie_problem_ncomp(P) -> int:
    return load().vie_problem_ncomp(P)


def vie_apply(P, x, y, precision: int, nrhs: int = 1, stream=None):
    need = _vec_bytes(P, None, nrhs, _elem(precision))
    px, py = _dev(x, need, "x"), _dev(y, need, "y")
    return _check(load().vie_apply(P, px, py, precision, nrhs, _stream(stream)))


def vie_apply_static(P, x, y, precision: int, nrhs: int = 1, stream=None):
    """vie_apply with the scratch in the library's fixed device array (allocates nothing)."""
    need = _vec_bytes(P, None, nrhs, _elem(precision))
    px, py = _dev(x, need, "x"), _dev(y, need, "y")
    return _check(load().vie_apply_static(P, px, py, precision, nrhs, _stream(stream)))


def vie_rhs_plane_wave(P, d, p, nrhs: int, rhs_out, stream=None):
    dd = _dvec(d)
    pp = None if p is None else _dvec(p)
    if len(dd) < 3 * nrhs or (pp is not None and len(pp) < 3 * nrhs):
        raise VieError(VIE_EINVAL, "vie_rhs_plane_wave: d and p need 3 values per right-hand side")
    out = _dev(rhs_out, _vec_bytes(P, None, nrhs, 16), "rhs_out")
    return _check(load().vie_rhs_plane_wave(P, dd, pp, nrhs, out, _stream(stream)))


def vie_solve(P, rhs, J, opts: SolveOpts, stream=None, allow_noconv=False):
    info = SolveInfo()
    allow = (VIE_OK, VIE_ENOCONV) if allow_noconv else (VIE_OK,)
    need = _vec_bytes(P, None, opts.nrhs, 16)
    pr, pj = _dev(rhs, need, "rhs"), _dev(J, need, "J")
    st = _check(load().vie_solve(P, pr, pj, ctypes.byref(opts), ctypes.byref(info), _stream(stream)), allow)
    return st, info


def vie_eval_scattered(P, J, field_out, nrhs: int = 1, stream=None):
    pj = _dev(J, _vec_bytes(P, None, nrhs, 16), "J")
    po = _dev(field_out, _vec_bytes(P, lambda sh: 6 if sh[2] == VIE_MAXWELL else 1, nrhs, 16), "field_out")
    return _check(load().vie_eval_scattered(P, pj, po, nrhs, _stream(stream)))


def vie_problem_bytes(kind: int, n: int, nrhs: int, restart: int, has_mu: int) -> int:
    return int(load().vie_problem_bytes(kind, n, nrhs, restart, has_mu))


def vie_problem_destroy(P):
    _SHAPES.pop(_key(P), None)
    return _check(load().vie_problem_destroy(P))


def vie_profile_begin(P, cap: int):
    return _check(load().vie_profile_begin(P, cap))


def vie_profile_end(P, nslots: int = 5):
    ms = (ctypes.c_double * nslots)()
    cnt = ctypes.c_int()
    _check(load().vie_profile_end(P, ms, nslots, ctypes.byref(cnt)))
    return list(ms), cnt.value


def vie_tune(P, precision: int, stream=None) -> int:
    v = ctypes.c_int()
    _check(load().vie_tune(P, precision, ctypes.byref(v), _stream(stream)))
    return v.value


def vie_last_error() -> str:
    return load().vie_last_error().decode()


# ------------------------------------------------------------ convenience


class Problem:
    """Owns a problem handle; tensors are torch CUDA tensors (complex128 / complex64)."""

    def __init__(self, kind, n, lo, hi, omega, eps, mu=None, stream=None):
        self.kind = KINDS[kind] if isinstance(kind, str) else kind
        self.n = n
        self._eps = eps  # keep alive until create returns (create synchronises)
        self.handle = vie_problem_create(self.kind, n, lo, hi, omega, eps, mu, stream)
        self.ncomp = vie_problem_ncomp(self.handle)

    def apply(self, x, y, precision=VIE_FP64, nrhs=1, stream=None):
        vie_apply(self.handle, x, y, precision, nrhs, stream)

    def rhs(self, d, p, nrhs, out, stream=None):
        vie_rhs_plane_wave(self.handle, d, p, nrhs, out, stream)

    def solve(self, rhs, J, tol=1e-10, restart=50, max_outer=50, max_inner=2000, inner_tol=1e-5,
              mode=VIE_SOLVE_FP64, nrhs=1, stream=None, allow_noconv=False, check_fp64=False):
        opts = SolveOpts(tol, restart, max_outer, max_inner, inner_tol, mode, nrhs, 1 if check_fp64 else 0)
        return vie_solve(self.handle, rhs, J, opts, stream, allow_noconv)

    def eval_scattered(self, J, out, nrhs=1, stream=None):
        vie_eval_scattered(self.handle, J, out, nrhs, stream)

    def tune(self, precision=VIE_FP32, stream=None) -> int:
        return vie_tune(self.handle, precision, stream)

    def close(self):
        if self.handle is not None:
            vie_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
