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


def declared_parameter_counts():
    """Parameter count of every function include/vie.h declares (comments stripped)."""
    src = open(os.path.join(ROOT, "include", "vie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(vie_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_the_header():
    """Every function the binding declares to ctypes takes as many arguments as the
    header says (a parameter added on one side only would shift every later one)."""
    entry.build()
    import paper_1805_04791_gb300 as vie

    counts = declared_parameter_counts()
    lib = vie.load()
    for name in vie.EXPORTED:
        assert name in counts, name
        assert len(getattr(lib, name).argtypes) == counts[name], name


def declared_struct_fields(name):
    """(type, field) pairs of `typedef struct { ... } name;` in include/vie.h, in order."""
    src = open(os.path.join(ROOT, "include", "vie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef\s+struct\s*\{([^}]*)\}\s*" + name + r"\s*;", src, flags=re.S)
    assert m, name
    return re.findall(r"(double|int)\s+([a-z_0-9]+)\s*;", m.group(1))


def test_binding_structs_match_the_header():
    """SolveOpts / SolveInfo have the header's fields, types and order (ctypes lays
    them out like the C compiler, so the same declaration gives the same offsets)."""
    import ctypes

    import paper_1805_04791_gb300 as vie

    ctype = {"double": ctypes.c_double, "int": ctypes.c_int}
    for cls, cname in ((vie.SolveOpts, "vie_solve_opts"), (vie.SolveInfo, "vie_solve_info")):
        declared = [(f, ctype[t]) for t, f in declared_struct_fields(cname)]
        assert [(f, t) for f, t in cls._fields_] == declared, cname
