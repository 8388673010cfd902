"""Host logic of bench.py that needs no GPU: the checksum that ties the
committed ncu traffic figures to the kernel sources follows their code and
ignores comments and layout."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_of_drops_comments_and_layout():
    src = "int a = 1; // one\n/* two\n lines */ int  b =\n 2;\n"
    assert bench.code_of(src) == "int a = 1; int b = 2;"
    assert bench.code_of("x /* a */ y /* b\n c */ z // d") == "x y z"


def test_code_of_keeps_code_changes():
    assert bench.code_of("int a = 1;") != bench.code_of("int a = 2;")
    assert bench.code_of("a // c\nb") == bench.code_of("a b // d")   # only the comments differ
    assert bench.code_of("a /* c */ + b") != bench.code_of("a - b")


def test_traffic_sha_is_the_committed_one_or_the_figure_is_null():
    sha = bench.traffic_sha()
    assert len(sha) == 16 and all(c in "0123456789abcdef" for c in sha)
    t = bench.committed_traffic("gather_vec_kernel")
    assert t is None or t > 0
