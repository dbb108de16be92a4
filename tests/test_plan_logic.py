"""Plan logic on the host (CPU): the passes, kernels, r x c splits and
workspace that moa_fft_plan chooses, read through moa_fft_estimate, which
describes a plan without a GPU.  The GPU tests check that a real plan makes
the same choices (test_gpu_autotune.py)."""
import ctypes

import pytest

TMA, NO_TMA = 1, 0


def pipe_col(logn, tw4, blk):
    """Name of the pipelined column kernel of a pass: at N = 4096 the
    two-columns-per-thread form, below it the four-column form."""
    return f"pipe_col2_kernel<{tw4},{blk}>" if logn == 12 else f"pipe_col_kernel<{logn},{tw4},{blk}>"


@pytest.fixture(scope="module")
def mf():
    from paper_0811_2535_gb300 import build, moafft
    build.build()
    return moafft


@pytest.mark.parametrize("L", range(1, 25))
@pytest.mark.parametrize("batch", [1, 3])
def test_1d_lifting(mf, L, batch):
    """n <= 4096: one on-chip tile (Sec. 3.6).  Larger n: lifted n = r*c with
    r = 2^floor(L/2) (Sec. 4.2, breakpoint of Sec. 4.8): an r-point column pass
    with the twiddle, then c-point rows stored transposed, through a
    workspace of one complex64 per element.  A pass of 1024..4096 points runs
    in a pipelined TMA kernel; when both do, the intermediate is blocked."""
    for tma in (TMA, NO_TMA):
        e = mf.estimate([1 << L], batch, tma=tma)
        if L <= 12:
            assert e == {"passes": 1, "split_r": 0, "split_c": 0, "workspace_bytes": 0,
                         "kernels": [f"row_pass_kernel<{L},0>"]}
            continue
        lr, lc = L // 2, L - L // 2
        assert (e["split_r"], e["split_c"]) == (1 << lr, 1 << lc)
        assert e["passes"] == 2 and e["workspace_bytes"] == 8 * batch << L
        pipe_r, pipe_c = tma == TMA and 10 <= lr <= 12, tma == TMA and 10 <= lc <= 12
        if pipe_r and pipe_c:
            assert e["kernels"] == [pipe_col(lr, 1, 1), pipe_col(lc, 0, 2)]
        else:
            assert e["kernels"] == [f"col_pass_kernel<{lr},1>",
                                    f"pipe_rowT_kernel<{lc}>" if pipe_c else f"row_pass_kernel<{lc},1>"]


def test_bench_workload_plans(mf):
    assert mf.estimate([1 << 24], tma=TMA)["kernels"] == ["pipe_col2_kernel<1,1>", "pipe_col2_kernel<0,2>"]
    assert mf.estimate([4096, 4096], tma=TMA) == {
        "passes": 2, "split_r": 0, "split_c": 0, "workspace_bytes": 0,
        "kernels": ["row_pass_kernel<12,0>", "pipe_col2_kernel<0,0>"]}
    assert mf.estimate([256, 256, 256], tma=TMA) == {
        "passes": 2, "split_r": 0, "split_c": 0, "workspace_bytes": 8 << 24,
        "kernels": ["plane3d_p1_kernel", "pipe_col2_kernel<0,3>"]}


@pytest.mark.parametrize("shape,batch", [((2, 2), 1), ((8, 16), 5), ((64, 32), 2), ((4096, 2), 1), ((2, 4096), 3),
                                         ((4, 8, 16), 2), ((256, 256, 256), 1), ((16, 4096, 2), 1)])
def test_multi_d_one_pass_per_axis(mf, shape, batch):
    """Eq. B.6 without the TMA kernels: the last axis as rows, then each other
    axis as a column pass, in place in the output (no workspace)."""
    e = mf.estimate(list(shape), batch, tma=NO_TMA)
    L = [s.bit_length() - 1 for s in shape]
    want = [f"row_pass_kernel<{L[-1]},0>"] + [f"col_pass_kernel<{L[a]},0>" for a in range(len(shape) - 2, -1, -1)]
    assert e["kernels"] == want and e["passes"] == len(shape)
    assert e["workspace_bytes"] == 0 and e["split_r"] == 0


def test_environment_overrides(mf, monkeypatch):
    monkeypatch.setenv("MOA_PIPE", "1")   # pipelined kernels, natural intermediate
    assert mf.estimate([1 << 24], tma=TMA)["kernels"] == ["pipe_col2_kernel<1,0>", "pipe_rowT_kernel<12>"]
    monkeypatch.setenv("MOA_PIPE", "0")   # generic kernels only, and one pass per axis in 3-D
    assert mf.estimate([1 << 24], tma=TMA)["kernels"] == ["col_pass_kernel<12,1>", "row_pass_kernel<12,1>"]
    assert mf.estimate([256, 256, 256], tma=TMA)["passes"] == 3
    monkeypatch.delenv("MOA_PIPE")
    monkeypatch.setenv("MOA_3D_TWO_PASS", "0")
    assert mf.estimate([256, 256, 256], tma=TMA)["kernels"] == [
        "row_pass_kernel<8,0>", "col_pass_kernel<8,0>", "col_pass_kernel<8,0>"]
    monkeypatch.delenv("MOA_3D_TWO_PASS")
    monkeypatch.setenv("MOA_SPLIT_LOG2R", "10")
    e = mf.estimate([1 << 22], tma=TMA)
    assert (e["split_r"], e["split_c"]) == (1024, 4096)
    assert e["kernels"] == ["pipe_col_kernel<10,1,1>", "pipe_col2_kernel<0,2>"]
    e = mf.estimate([1 << 24], tma=TMA)   # c would be 2^14: out of range, default split kept
    assert (e["split_r"], e["split_c"]) == (4096, 4096)
    monkeypatch.delenv("MOA_SPLIT_LOG2R")
    monkeypatch.setenv("MOA_LIFT3", "1")   # three-level lift: r = 256, rows of 2^16 as 256 x 256
    e = mf.estimate([1 << 24], tma=TMA)
    assert e["kernels"] == ["col_pass_kernel<8,1>", "lift3_kernel<8,8>"]
    assert (e["split_r"], e["split_c"]) == (256, 1 << 16)
    assert mf.estimate([1 << 20], tma=TMA)["kernels"][1] == "pipe_col_kernel<10,0,2>"   # below 2^21: no lift3


def test_tensor_core_plans(mf, monkeypatch):
    assert mf.estimate([4096], 4, dtype=1, tma=NO_TMA)["kernels"] == ["tc_umma_kernel<0,12>"]
    assert mf.estimate([256], 4, dtype=2, tma=NO_TMA)["kernels"] == ["tc_umma_kernel<1,8>"]
    monkeypatch.setenv("MOA_TC_KERNEL", "sync")
    assert mf.estimate([4096], 1, dtype=2, tma=TMA)["kernels"] == ["tc_row_kernel<1,12>"]


def test_estimate_rejects_what_plan_rejects(mf):
    L = mf.lib()

    def code(shape, batch=1, dtype=0, tma=1, buf=None, buflen=0):
        arr = (ctypes.c_int64 * max(1, len(shape)))(*shape)
        return L.moa_fft_estimate(arr if shape else None, len(shape), batch, dtype, tma,
                                  None, None, None, None, buf, buflen)

    assert code([1 << 24]) == 0
    assert code([12]) == 2 and code([1]) == 2 and code([8, 6]) == 2        # not a power of two >= 2
    assert code([1 << 25]) == 0 and code([8192, 2]) == 0                  # lifted further / a long axis
    assert code([1 << 31]) == 3 and code([1 << 25, 2]) == 3               # beyond the supported sizes
    assert code([1 << 24], batch=128) == 3                                # 2^31 elements
    assert code([64], dtype=1) == 3                                       # tensor cores: 256 or 4096 only
    assert code([8], batch=0) == 1 and code([8], dtype=7) == 1 and code([2, 2, 2, 2]) == 1
    assert code([]) == 1                                                  # no shape
    assert code([8], tma=2) == 1 and code([8], tma=-2) == 1
    assert code([8], buf=None, buflen=16) == 1                            # NULL buffer with a length
    small = ctypes.create_string_buffer(8)                                # truncated, NUL-terminated
    assert code([1 << 24], buf=small, buflen=8) == 0 and small.value == b"pipe_co"
    with pytest.raises(mf.MoaError):
        mf.estimate([3])


@pytest.mark.parametrize("L", range(25, 31))
@pytest.mark.parametrize("tma", [TMA, NO_TMA])
def test_1d_beyond_2_24(mf, L, tma):
    """n > 2^24: n = r1*r2*c (Sec. 4.2 applied twice; c = 2^ceil(L/3), r = r1*r2
    balanced): an r2-point column pass with the twiddle of the r-point
    transform, an r1-point column pass storing row k1s + r2*k1f with the
    four-step twiddle, then the c-point rows stored transposed; in -> out ->
    workspace -> out."""
    e = mf.estimate([1 << L], 1, tma=tma)
    lc = (L + 2) // 3
    lr = L - lc
    lr1, lr2 = (lr + 1) // 2, lr - (lr + 1) // 2
    assert (e["passes"], e["split_r"], e["split_c"], e["workspace_bytes"]) == (3, 1 << lr, 1 << lc, 8 << L)
    row = f"pipe_rowT_kernel<{lc}>" if tma == TMA and lc >= 10 else f"row_pass_kernel<{lc},1>"
    assert e["kernels"] == [f"col_pass_kernel<{lr2},1>", f"col_pass_kernel<{lr1},1>", row]


@pytest.mark.parametrize("shape,batch,kernels", [
    ((8192, 2048), 1, ["row_pass_kernel<11,0>", "col_pass_kernel<6,1>", "col_pass_kernel<7,0>"]),
    ((2048, 8192), 1, ["col_pass_kernel<6,1>", "row_pass_kernel<7,1>", "pipe_col_kernel<11,0,0>"]),
    ((16, 8192, 8), 2, ["row_pass_kernel<3,0>", "col_pass_kernel<6,1>", "col_pass_kernel<7,0>",
                        "col_pass_kernel<4,0>"]),
    ((1 << 20, 2), 1, ["row_pass_kernel<1,0>", "col_pass_kernel<10,1>", "col_pass_kernel<10,0>"]),
    ((8192, 8192), 1, ["col_pass_kernel<6,1>", "row_pass_kernel<7,1>", "col_pass_kernel<6,1>",
                       "col_pass_kernel<7,0>"])])
def test_multi_d_long_axes(mf, shape, batch, kernels):
    """Eq. B.6 with an axis longer than 4096: that axis lifted L = L1*L2
    (L2 = 2^floor(l/2) points over the slow half with the twiddle, then L1
    points over the fast half, the last axis's second half as a transposed
    row pass), the other axes one pass each; every pass through the
    workspace, the last into the output."""
    e = mf.estimate(list(shape), batch, tma=TMA)
    n = batch
    for s_ in shape:
        n *= s_
    assert e["kernels"] == kernels
    assert (e["passes"], e["workspace_bytes"]) == (len(kernels), 8 * n)


def test_four_column_kernel_on_request():
    """MOA_COL2=0 (read once per process, so checked in a child process):
    the N = 4096 column passes name the four-column kernel."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_0811_2535_gb300 import moafft\n"
            "print(moafft.estimate([1 << 24], tma=1)['kernels'], moafft.estimate([256] * 3, tma=1)['kernels'])\n") % root
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300,
                         env=dict(os.environ, MOA_COL2="0"))
    assert res.returncode == 0, res.stderr
    assert res.stdout.strip() == ("['pipe_col_kernel<12,1,1>', 'pipe_col_kernel<12,0,2>'] "
                                  "['plane3d_p1_kernel', 'pipe_col_kernel<12,0,3>']")


@pytest.mark.parametrize("v", [1, 2, 3])
def test_radix_schedule_override(mf, v, monkeypatch):
    """MOA_SCHED picks the radix schedule of the generic passes (Sec. 4.8:
    any factorisation of the in-register stages): 1 = small radix last
    (2^9..2^11), 2 = radix-8 stages (2^7..2^12), 3 = the warp-shuffle kernel
    for natural-order rows of 2^7..2^9 points whose blocks are whole warps.
    A pass for which the schedule does not exist, and every pipelined or
    fused pass, keeps its own."""
    monkeypatch.setenv("MOA_SCHED", str(v))
    ok = {1: range(9, 12), 2: range(7, 13), 3: range(7, 10)}[v]
    for L in range(1, 13):
        for batch in (1, 64):
            k = mf.estimate([1 << L], batch, tma=TMA)["kernels"]
            threads = (1 << max(L - 4, 0)) << min(12 - L, (batch - 1).bit_length()) if L <= 12 else 0
            if L in ok and (v != 3 or threads % 32 == 0):
                assert k == [f"row_warp_kernel<{L}>" if v == 3 else f"row_pass_kernel<{L},0,{v}>"], (L, batch)
            else:
                assert k == [f"row_pass_kernel<{L},0>"], (L, batch)
    # the pipelined N = 4096 passes and the two-pass 3-D form keep their kernels
    assert mf.estimate([1 << 24], tma=TMA)["kernels"] == ["pipe_col2_kernel<1,1>", "pipe_col2_kernel<0,2>"]
    assert mf.estimate([256, 256, 256], tma=TMA)["kernels"] == ["plane3d_p1_kernel", "pipe_col2_kernel<0,3>"]
    # generic lifted passes: column pass with the twiddle and transposed rows
    k = mf.estimate([1 << 18], tma=NO_TMA)["kernels"]
    if v == 3:   # transposed rows and column passes keep schedule 0
        assert k == ["col_pass_kernel<9,1>", "row_pass_kernel<9,1>"]
    else:
        assert k == [f"col_pass_kernel<9,1,{v}>", f"row_pass_kernel<9,1,{v}>"]
