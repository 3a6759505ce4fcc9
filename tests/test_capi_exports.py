"""The C-ABI library builds, loads and exports every function include/vie.h declares (no GPU needed)."""
import ctypes
import os
import re

import __graft_entry__ as entry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+(vie_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("vie_problem_create", "vie_apply", "vie_solve", "vie_eval_scattered", "vie_rhs_plane_wave",
                     "vie_problem_destroy", "vie_problem_bytes", "vie_last_error", "vie_problem_ncomp"):
        assert required in names


def test_library_exports_every_declared_symbol():
    entry.build()
    import paper_1805_04791_gb300 as vie

    lib = ctypes.CDLL(vie.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(vie.EXPORTED) <= set(declared_functions())


def test_memory_estimate_is_monotone():
    entry.build()
    import paper_1805_04791_gb300 as vie

    a = vie.vie_problem_bytes(vie.VIE_HELMHOLTZ, 64, 1, 50, 0)
    b = vie.vie_problem_bytes(vie.VIE_HELMHOLTZ, 128, 1, 50, 0)
    c = vie.vie_problem_bytes(vie.VIE_MAXWELL, 128, 1, 50, 1)
    assert 0 < a < b < c
