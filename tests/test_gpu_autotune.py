"""Plan-time autotuner (GPU): it times the admissible r x c splits of a
lifted 1-D transform and its three-level lift, the pipelined or generic
strided kernels, the tile size of the generic passes, the two-pass or
per-axis form of 256^3 arrays, and the per-length split of a batched plan;
it keeps the fastest, records the choice in its cache file and reuses it;
results stay within the parity tolerance whatever it picks, and the plan
states its choice (moa_fft_plan_choice)."""
import os
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 2e-6


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0811_2535_gb300 import build, moafft
    build.build()
    import oracle
    oracle.build()
    return torch, moafft, oracle


def test_autotuned_split_is_cached_and_correct(env, tmp_path, monkeypatch):
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("MOA_TUNE_CACHE", str(cache))
    monkeypatch.setenv("MOA_AUTOTUNE", "1")
    for k in ("MOA_SPLIT_LOG2R", "MOA_PIPE", "MOA_BATCH_LOG2R"):
        monkeypatch.delenv(k, raising=False)
    n = 1 << 19          # a size not planned elsewhere in this process
    t0 = time.perf_counter()
    plan = moafft.Plan([n], 3, -1)
    t_first = time.perf_counter() - t0
    info = plan.info()
    text = cache.read_text()
    line = [ln for ln in text.splitlines() if ":plan:1:524288:3:ssssss " in ln]
    assert len(line) == 1, text
    lr, pipe, lift3, tile, two, sched = (int(v) for v in line[0].split()[1:7])
    assert lift3 == 0          # the three-level lift is a candidate from 2^21 on
    assert info["split_r"] == 1 << lr and 7 <= lr <= 12
    assert tile in (11, 12, 13) and two == -1 and sched in (-1, 1, 2, 3)
    assert "autotuned" in plan.choice() and ("r=%d" % (1 << lr)) in plan.choice()
    x = inputs.uniform((3, n), 77)
    y = plan.exec(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.fft_radix2(x.astype(np.complex128), -1)
    err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= TOL
    plan.destroy()
    t0 = time.perf_counter()
    again = moafft.Plan([n], 3, -1)       # served from the cache: no timing runs
    t_second = time.perf_counter() - t0
    assert again.info()["split_r"] == info["split_r"]
    assert "from the cache" in again.choice()
    assert t_second < t_first
    again.destroy()


def test_autotuned_batched_plan(env, tmp_path, monkeypatch):
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("MOA_TUNE_CACHE", str(cache))
    monkeypatch.setenv("MOA_AUTOTUNE", "1")
    monkeypatch.delenv("MOA_BATCH_LOG2R", raising=False)
    lengths = [1 << k for k in (14, 9, 16, 13, 6, 15, 12)]
    vecs = [inputs.uniform(n, 80 + i) for i, n in enumerate(lengths)]
    plan = moafft.BatchedPlan(lengths, -1)
    # the entry is keyed by the histogram of log2 lengths; the cache file also
    # holds entries of plans made earlier in this process
    hist = [0] * 17
    for n in lengths:
        hist[n.bit_length() - 1] += 1
    key = ":batched2:" + ",".join(str(h) for h in hist[1:]) + " "
    line = [ln for ln in cache.read_text().splitlines() if key in ln]
    assert len(line) == 1, cache.read_text()
    offsets = [int(v) for v in line[0].split()[1:5]]
    assert all(o in (-1, 0, 1) for o in offsets)
    assert "autotuned" in plan.choice() and "2^16:%d" % offsets[3] in plan.choice()
    x = torch.from_numpy(np.concatenate(vecs)).cuda()
    y = plan.exec(x).cpu().numpy()
    for o, n, v in zip(plan.offsets(), lengths, vecs):
        ref = oracle.fft_radix2(v.astype(np.complex128), -1)
        assert np.linalg.norm(y[o:o + n] - ref) / np.linalg.norm(ref) <= TOL
    plan.destroy()


def test_plan_log(env, tmp_path):
    """MOA_LOG=1: the autotuner's timed candidates and the chosen plan are
    written to stderr (checked in a child process, whose stderr is captured)."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_0811_2535_gb300 import moafft\n"
            "p = moafft.Plan([1 << 17], 2, -1); p.destroy()\n"
            "q = moafft.Plan([64, 32], 1, 1); q.destroy()\n") % root
    envv = dict(os.environ, MOA_LOG="1", MOA_AUTOTUNE="1", MOA_TUNE_CACHE=str(tmp_path / "tune.txt"))
    for k in ("MOA_SPLIT_LOG2R", "MOA_PIPE", "MOA_BATCH_LOG2R", "MOA_LIFT3"):
        envv.pop(k, None)
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=envv, timeout=300)
    assert res.returncode == 0, res.stderr
    lines = [ln for ln in res.stderr.splitlines() if ln.startswith("moafft: ")]
    cands = [ln for ln in lines if ln.startswith("moafft: autotune candidate ")]
    # 1-D 2^17: splits 2^5..2^12, with pipelined and generic kernels and three tiles
    assert sum("col_pass_kernel<" in ln or "pipe_col" in ln for ln in cands) >= 8, lines
    # 2-D 64 x 32: the tile sizes of its two generic passes
    assert any("row_pass_kernel<5,0>/" in ln and "col_pass_kernel<6,0>/" in ln for ln in cands), lines
    plan_lines = [ln for ln in lines if ln.startswith("moafft: plan ")]
    assert len(plan_lines) == 2, lines
    assert "131072 batch 2 sign -1" in plan_lines[0] and "autotuned" in plan_lines[0]
    assert "64x32 batch 1 sign +1" in plan_lines[1] and "row_pass_kernel<5,0> -> col_pass_kernel<6,0>" in plan_lines[1]
    assert "autotuned" in plan_lines[1]


@pytest.mark.parametrize("shape,batch", [((1 << 22,), 1), ((1 << 12,), 16), ((4096, 4096), 1),
                                         ((512, 1024), 2), ((256, 256, 256), 1), ((64, 32, 128), 2)])
def test_every_tuned_plan_kind_matches_oracle(env, shape, batch, tmp_path, monkeypatch):
    """Lifted 1-D, batched 1-D rows, 2-D and 3-D plans, each tuned from an
    empty cache: the chosen plan is stated and its output matches the FP64
    oracle."""
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    monkeypatch.setenv("MOA_TUNE_CACHE", str(tmp_path / "tune.txt"))
    monkeypatch.setenv("MOA_AUTOTUNE", "1")
    for k in ("MOA_SPLIT_LOG2R", "MOA_PIPE", "MOA_TILE_LOG2", "MOA_3D_TWO_PASS", "MOA_LIFT3"):
        monkeypatch.delenv(k, raising=False)
    plan = moafft.Plan(list(shape), batch, -1)
    assert "autotuned" in plan.choice()
    x = inputs.uniform((batch,) + tuple(shape), 90 + len(shape))
    y = plan.exec(torch.from_numpy(x.reshape(-1)).cuda()).cpu().numpy().reshape(batch, -1)
    assert plan.status() == 0
    plan.destroy()
    x64 = x.astype(np.complex128)
    ref = (oracle.fft_radix2(x64, -1) if len(shape) == 1 else oracle.fft_nd(x64, len(shape), -1)).reshape(batch, -1)
    err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= TOL


@pytest.mark.parametrize("shape,batch,dtype", [((1 << 24,), 1, 0), ((1 << 25,), 1, 0), ((8192, 2048), 1, 0),
                                               ((2048, 8192), 2, 0), ((1 << 19,), 2, 0), ((1 << 13,), 3, 0),
                                               ((1 << 10,), 4, 0), ((4096, 4096), 1, 0), ((256, 256, 256), 1, 0),
                                               ((8, 16, 32), 2, 0), ((4096,), 8, 1), ((256,), 8, 2)])
def test_estimate_matches_the_plan(env, shape, batch, dtype, monkeypatch):
    """moa_fft_estimate, asking the driver (tma = -1), describes exactly the
    plan moa_fft_plan builds with the autotuner off."""
    _, moafft, _ = env
    monkeypatch.setenv("MOA_AUTOTUNE", "0")
    e = moafft.estimate(list(shape), batch, dtype=dtype, tma=-1)
    plan = moafft.Plan(list(shape), batch, -1, dtype)
    info = plan.info()
    kernels = [plan.pass_info(i)["kernel"] for i in range(info["passes"])]
    plan.destroy()
    assert e["kernels"] == kernels
    assert (e["passes"], e["split_r"], e["split_c"], e["workspace_bytes"]) == \
        (info["passes"], info["split_r"], info["split_c"], info["workspace_bytes"])


@pytest.mark.parametrize("L,batch", [(9, 4096), (11, 1024)])
def test_autotuner_times_radix_schedules(env, tmp_path, monkeypatch, capfd, L, batch):
    """The search covers the radix schedule of the generic passes (Sec. 4.8:
    any factorisation of the in-register stages): small radix first or last,
    radix-8 stages, and for 2^7..2^9-point rows the warp-shuffle kernel.
    MOA_LOG=1 lists every timed candidate; the plan kept matches the oracle."""
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    monkeypatch.setenv("MOA_TUNE_CACHE", str(tmp_path / "tune.txt"))
    monkeypatch.setenv("MOA_AUTOTUNE", "1")
    monkeypatch.setenv("MOA_LOG", "1")
    for k in ("MOA_SCHED", "MOA_PIPE"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setenv("MOA_TILE_LOG2", "12")   # 256-thread blocks, which the warp-shuffle kernel takes
    n = 1 << L
    plan = moafft.Plan([n], batch, -1)
    err_text = capfd.readouterr().err
    timed = [ln for ln in err_text.splitlines() if "autotune candidate" in ln]
    want = [f"row_pass_kernel<{L},0>", f"row_pass_kernel<{L},0,1>", f"row_pass_kernel<{L},0,2>"]
    if L <= 9:
        want.append(f"row_warp_kernel<{L}>")
    for w in want:
        assert any(w + "/" in ln for ln in timed), (w, timed)
    x = inputs.uniform((batch, n), 90 + L)
    y = plan.exec(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.fft_radix2(x.astype(np.complex128), -1)
    err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= TOL
    plan.destroy()
