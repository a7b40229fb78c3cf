"""bench.py's key for the recorded ncu traffic of the pass groups: it hashes
the code of the kernel sources, so a comment or whitespace edit keeps it
and a code edit changes it (a changed kernel then reports no traffic); and
the recorded values are plausible DRAM traffic for a group launch."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_comments_and_whitespace_do_not_count():
    code = "int f(int x) {\n  return x + 1;  // add one\n}\n"
    assert bench.kernel_code(code) == bench.kernel_code("/* doc\n   block */ int f(int  x) { return x + 1; }")
    assert bench.kernel_code(code) != bench.kernel_code(code.replace("x + 1", "x + 2"))
    # a "//" inside a block comment and a block comment spanning lines
    assert bench.kernel_code("a; /* x // y\n z */ b;") == "a; b;"


def test_recorded_traffic_is_plausible():
    """Every recorded entry lies between 95 % and 100 % of the algorithmic
    bytes of a whole group on 2^28 amplitudes (reads once, writes once; the
    last tiles' writes still in L2 at the end of a launch)."""
    assert bench.NCU_TRAFFIC
    for (key, dtype), traffic in bench.NCU_TRAFFIC.items():
        assert len(key) == 16
        amp = 8 if dtype == "c64" else 16
        assert 0.95 * 2 * 2 ** 28 * amp < traffic < 2 * 2 ** 28 * amp, (key, dtype, traffic)
