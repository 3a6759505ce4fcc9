"""FP64 CPU oracle for the FFT-accelerated volume-integral-equation operators.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The product library never calls it and shares no
code with it; the two meet only in the seeded input generators of
``vie_inputs`` (which hold none of the method's arithmetic).

The oracle is deliberately plain: numpy/scipy in float64/complex128, one
library FFT as a step where the definition is a discrete Fourier sum, no
blocking, fusion or reordering beyond what the definitions state.  Every
function cites the passage of Imbert-Gerard, Vico, Greengard, Ferrando,
"Integral equation methods for electrostatics, acoustics and electromagnetics
in smoothly varying, anisotropic media" (arXiv:1805.04791) that it follows.

Modules
-------
``greens``     truncated free-space Green's function transforms (Sec. 5, a-c).
``discrete``   the discrete convolution kernels on the uniform grid.
``operators``  H tensors, the operators I+B+K of Eqs. (eq:intLap), (eq:intH),
               (eq:intM), right-hand sides and scattered fields.
``solvers``    Neumann series, restarted GMRES, Bi-CGStab, dense LU.

Pins: every function is checked in ``tests/test_oracle_*.py`` against closed
forms, independent quadrature, brute-force sums and theorems of the paper.
"""

from . import greens, discrete, operators, solvers  # noqa: F401
