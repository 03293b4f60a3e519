"""bench.py's host-side helpers (no GPU): the code-only source hash that
decides whether the committed ncu traffic still applies, and the fixed
algorithmic flop count."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_only_drops_comments_and_layout_but_keeps_literals():
    a = 'int f(int x) {  // twice\n  return 2 * x; /* doubled */ }\nconst char* s = "a // b /* c */";\n'
    b = 'int f(int x) { return 2 * x; }\n// moved\nconst char* s = "a // b /* c */";'
    assert bench.code_only(a) == bench.code_only(b)
    assert '"a // b /* c */"' in bench.code_only(a)
    assert bench.code_only("char q = '\"'; int y; // z") == "char q = '\"'; int y;"
    assert bench.code_only(a) != bench.code_only(a.replace("2 * x", "3 * x"))


def test_fixed_flop_count():
    """The algorithmic count depends on the iterations a run takes, never on
    the build: p2r 600 + 50 per iteration, p2z 580."""
    assert bench.flops_p2r(1.0) == 650.0
    assert bench.flops_p2r(2.0) == 700.0
    assert bench.FLOPS_P2Z == 580.0
    assert bench.fp32_peak_tflops(2070.0, 152) == 152 * 128 * 2 * 2070e6 / 1e12
