"""bench.py's host-side helpers (no GPU): the code-only source hash that
decides whether the committed ncu traffic still applies, and the flop count
of the straight-line start."""
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


def test_flop_count_of_the_straight_line_start():
    assert bench.flops_p2r_line(2.007) == bench.FLOPS_P2R_LINE
    assert bench.flops_p2r_line(1.0) < bench.FLOPS_P2R_LINE
