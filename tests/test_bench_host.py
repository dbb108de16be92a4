"""Host-side helpers of the benchmark (CPU): the reference arm's sample
shapes and the kernel-source hash that ties committed DRAM counters to the
code they were taken on."""
import math
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


@pytest.mark.parametrize("s", range(0, 12))
def test_reference_shapes_are_valid_and_scaled(s):
    import bench
    shapes = bench.reference_shapes(s)
    assert len(shapes) == 3 and [len(sh) for sh in shapes] == [1, 2, 3]
    for sh in shapes:
        for d in sh:
            assert d >= 2 and d & (d - 1) == 0, (s, sh)
        assert math.prod(sh) == (1 << 24) >> s, (s, sh)


def test_kernel_hash_ignores_comments_only():
    import bench
    code = "int f(int a) { return a + 1; }\n"
    assert bench._code_only("// note\n" + code + "/* a\n b */\n\n") == bench._code_only(code)
    assert bench._code_only(code) != bench._code_only(code.replace("+ 1", "+ 2"))
    h = bench.kernel_src_hash("pipe_col_kernel<12,1,1>")
    assert len(h) == 16 and h == bench.kernel_src_hash("pipe_col_kernel<12,0,2>")
    assert h != bench.kernel_src_hash("row_pass_kernel<12,0>")
