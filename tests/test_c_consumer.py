"""A plain C99 program uses the library through include/vie.h alone (no GPU needed).

The boundary is a C ABI: the header must compile as C (and C++), and a C caller
linked against the shared library must get the same answers as the Python
binding.  The calls exercised need no device: the memory estimate, argument
refusals that return before any CUDA call, and the thread-local error message.
"""
import os
import shutil
import subprocess

import pytest

import __graft_entry__ as entry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SOURCE = r"""
#include <stdio.h>
#include <string.h>
#include "vie.h"

int main(void) {
  /* memory estimate for admission: Helmholtz 64^3 and 128^3, Maxwell with mu 128^3 */
  printf("%zu %zu %zu\n", vie_problem_bytes(VIE_HELMHOLTZ, 64, 1, 50, 0),
         vie_problem_bytes(VIE_HELMHOLTZ, 128, 1, 50, 0), vie_problem_bytes(VIE_MAXWELL, 128, 1, 50, 1));
  /* refusals that return before touching a device */
  vie_problem* P = (vie_problem*)0;
  vie_status s1 = vie_problem_create(VIE_LAPLACE, 3, -1.0, 1.0, 0.0, (const void*)0, (const void*)0, (void*)0, &P);
  const char* m1 = vie_last_error();
  char msg1[256];
  strncpy(msg1, m1, sizeof msg1 - 1);
  msg1[sizeof msg1 - 1] = 0;
  vie_status s2 = vie_apply((vie_problem*)0, (const void*)0, (void*)0, VIE_FP64, 1, (void*)0);
  printf("%d %d %d\n", (int)s1, (int)s2, P == (vie_problem*)0);
  printf("%s\n%s\n", msg1, vie_last_error());
  return 0;
}
"""


def test_c99_program_links_and_matches_the_binding(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    entry.build()
    import paper_1805_04791_gb300 as vie

    src = tmp_path / "consumer.c"
    exe = tmp_path / "consumer"
    src.write_text(C_SOURCE)
    libdir = os.path.dirname(vie.LIB_PATH)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-lvie_gb300", f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    sizes = [int(v) for v in out[0].split()]
    assert sizes == [vie.vie_problem_bytes(vie.VIE_HELMHOLTZ, 64, 1, 50, 0),
                     vie.vie_problem_bytes(vie.VIE_HELMHOLTZ, 128, 1, 50, 0),
                     vie.vie_problem_bytes(vie.VIE_MAXWELL, 128, 1, 50, 1)]
    s1, s2, untouched = (int(v) for v in out[1].split())
    assert s1 == vie.VIE_EINVAL and s2 == vie.VIE_EINVAL and untouched == 1
    assert "n must be" in out[2]       # the create refusal names the size rule
    assert "vie_apply" in out[3]       # the last error is the latest call's


def test_header_compiles_as_cpp(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "consumer.cpp"
    src.write_text('#include "vie.h"\nint main() { return vie_problem_bytes(VIE_LAPLACE, 8, 1, 10, 0) == 0; }\n')
    subprocess.run([gxx, "-std=c++17", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                    "-I", os.path.join(ROOT, "include"), str(src)], check=True)
