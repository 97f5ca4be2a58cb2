"""Host logic of bench.py that decides whether a committed ncu traffic figure
still describes the kernel: the sources are compared without their comments,
so an edited comment keeps the figure and an edited line of code drops it
(the bench then reports the traffic as null)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_comments_are_dropped_but_literals_kept():
    src = ('int a = 1; // a comment\n/* block\n comment */ const char* s = "x//y /* z */";\n'
           "char c = '/'; char q = '\\''; int b = a / 2; // end")
    assert bench.code_only(src) == ('int a = 1; const char* s = "x//y /* z */"; char c = \'/\'; '
                                    "char q = '\\''; int b = a / 2;")


def test_code_changes_are_seen_comment_changes_are_not():
    base = "__global__ void k(int* p) {\n  // store one\n  *p = 1;\n}\n"
    assert bench.code_only(base) == bench.code_only(base.replace("store one", "store a one"))
    assert bench.code_only(base) == bench.code_only(base.replace("\n  *p", "\n\n    *p"))
    assert bench.code_only(base) != bench.code_only(base.replace("= 1", "= 2"))

