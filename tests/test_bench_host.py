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


def test_template_step_small_workload_equals_oracle():
    """The CPU comparison leg on a small step: every output equals the
    sequential oracle's, and the 1-D processor count stays a power of two
    with m * m <= n."""
    import bench
    secs, threads, m, same = bench.template_step([(1 << 12,), (64, 32), (16, 8, 4)], 1, reps=1)
    assert same and secs > 0 and threads >= 1
    assert m >= 1 and (m & (m - 1)) == 0 and m <= threads and m * m <= 1 << 12


def test_host_cpu_record():
    import bench
    h = bench.host_cpu()
    assert set(h) == {"machine", "model", "nproc"} and h["nproc"] >= 1 and h["machine"]
