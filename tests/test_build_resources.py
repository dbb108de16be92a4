"""Register and spill budget of the kernels (CPU: nvcc and ptxas only, no GPU).

Every kernel's registers, stack frame and spills as ptxas reports them for
sm_103a (-Xptxas -v, the build's own flags).  The budget the kernels are
designed to:
  * no kernel spills, except the batched persistent kernel (32 bytes, the
    price of four resident blocks per SM at 64 registers) and the
    small-radix-last schedule of 512-point rows, an autotuner candidate
    (under 128 bytes);
  * the two-column N = 4096 pipelined kernel fits its 512 threads in the
    register file (at most 128 registers a thread);
  * the generic pass kernels, launched with up to 1024 threads, and the
    warp-shuffle rows stay within 64 registers."""
import concurrent.futures as cf
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

UNITS = ["pass_kernels.cu", "pipe_kernels.cu", "batched.cu", "tc_umma.cu", "lift3.cu"]


def ptxas_report(unit, tmp):
    from paper_0811_2535_gb300 import build
    src = os.path.join(ROOT, "paper_0811_2535_gb300", "csrc", unit)
    cmd = [build.nvcc()] + build.ARCH + build.NVCC_FLAGS + ["-Xptxas", "-v", "-c", src, "-o",
                                                             os.path.join(tmp, unit + ".o")]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    kernels, cur = {}, None
    for line in res.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            cur = m.group(1)
            kernels[cur] = {}
            continue
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and cur:
            kernels[cur]["stack"], kernels[cur]["spill_st"], kernels[cur]["spill_ld"] = map(int, m.groups())
            continue
        m = re.search(r"Used (\d+) registers", line)
        if m and cur:
            kernels[cur]["regs"] = int(m.group(1))
    names = subprocess.run(["c++filt"], input="\n".join(kernels), capture_output=True, text=True).stdout.split("\n")
    return {n: kernels[k] for n, k in zip(names, kernels)}


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("ptxas"))
    with cf.ThreadPoolExecutor(len(UNITS)) as ex:
        parts = list(ex.map(lambda u: ptxas_report(u, tmp), UNITS))
    out = {}
    for p in parts:
        out.update(p)
    return out


def allowed_spill(name):
    if "batched_kernel" in name:
        return 32
    if re.search(r"row_pass_kernel<9, (true|false), 1>", name):
        return 128
    return 0


def test_every_kernel_reported(report):
    for fam in ("pipe_col2_kernel", "pipe_col_kernel", "pipe_rowT_kernel", "row_pass_kernel", "col_pass_kernel",
                "row_warp_kernel", "plane3d_p1_kernel", "batched_kernel", "tc_umma_kernel", "lift3_kernel"):
        assert any(fam + "<" in n or fam + "(" in n for n in report), fam
    assert all("regs" in v and "spill_st" in v for v in report.values())


def test_spills_within_budget(report):
    over = {n: v["spill_st"] for n, v in report.items() if v["spill_st"] > allowed_spill(n)}
    assert not over, over


def test_register_budgets(report):
    for n, v in report.items():
        if "pipe_col2_kernel" in n:
            assert v["regs"] <= 128, (n, v)
        if re.search(r"(row_pass_kernel|col_pass_kernel|row_warp_kernel)<", n):
            assert v["regs"] <= 64, (n, v)
