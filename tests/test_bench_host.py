"""Host-side pieces of bench.py (no GPU): the algorithmic bytes of the five passes.

The roofline reported by bench.py divides these bytes by measured pass times, so
they are checked against the buffers of the documented layout: x and y are
c N values, the x-pass output A is [c][n][n][2n] (2c N), the y-pass output B is
[c][n][2n][2n] (4c N, the z planes >= n are never stored), H has 6 N entries and
each of the 6 kernel octants (n+1)^3.
"""
import bench


def layout_bytes(n, c, esz):
    N = n ** 3
    x = y = c * N
    A = c * n * n * (2 * n)
    B = c * n * (2 * n) * (2 * n)
    H = 6 * N
    K = 6 * (n + 1) ** 3
    passes = [x + A, A + B, B + K + B, B + A, A + x + H + y]
    return [v * esz for v in passes]


def test_pass_bytes_follow_the_layout():
    for n, c in ((32, 3), (128, 3), (64, 6)):
        for esz in (8, 16):
            assert bench.algorithmic_bytes(n, c, esz) == layout_bytes(n, c, esz)


def test_quoted_figures_for_the_bench_workload():
    b = bench.algorithmic_bytes(128, 3, 8)  # Helmholtz 128^3, FP32 complex
    assert round(b[2] / 1e6, 1) == 505.7  # the z pass (the roofline's kernel)
    assert round(sum(b) / 1e9, 2) == 1.56  # one apply
