"""Batched uneven transforms in one persistent launch (GPU): every
transform against the FP64 oracle, CUDA-graph capture and replay, every
in-block split of the large transforms, the full 4096-transform workload."""
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


def run_batched(env, lengths, vecs, sign, graph=False):
    torch, moafft, _ = env
    plan = moafft.BatchedPlan(lengths, sign)
    x = torch.from_numpy(np.concatenate(vecs)).cuda()
    out = torch.empty_like(x)
    if graph:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            plan.exec(x, out, stream=s)          # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            plan.exec(x, out, stream=torch.cuda.current_stream())
        out.zero_()
        g.replay()
        first = out.clone()
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(first, out)
    else:
        plan.exec(x, out)
    y = out.cpu().numpy()
    assert plan.status() == 0
    offs = plan.offsets()
    plan.destroy()
    return [y[o:o + n] for o, n in zip(offs, lengths)]


def check(env, lengths, vecs, ys, sign):
    _, _, oracle = env
    worst = 0.0
    for n, x, y in zip(lengths, vecs, ys):
        ref = oracle.fft_radix2(x.astype(np.complex128), sign)
        err = np.linalg.norm(y.astype(np.complex128) - ref) / np.linalg.norm(ref)
        worst = max(worst, err)
        assert err <= TOL, (n, err)
    return worst


@pytest.mark.parametrize("sign", [-1, 1])
def test_mixed_lengths_every_size(env, sign):
    from paper_0811_2535_gb300 import inputs
    rng = np.random.default_rng(41)
    lengths = [1 << int(k) for k in rng.permutation(np.repeat(np.arange(1, 17), 3))]
    vecs = [inputs.uniform(n, 100 + i) for i, n in enumerate(lengths)]
    check(env, lengths, vecs, run_batched(env, lengths, vecs, sign), sign)


def test_many_small_of_one_size_and_ragged_groups(env):
    from paper_0811_2535_gb300 import inputs
    lengths = [64] * 67 + [2] * 300 + [4096] * 3 + [16] * 257
    vecs = [inputs.uniform(n, 500 + i) for i, n in enumerate(lengths)]
    check(env, lengths, vecs, run_batched(env, lengths, vecs, -1), -1)


def test_graph_capture_and_replay(env):
    from paper_0811_2535_gb300 import inputs
    lengths = [1 << k for k in (16, 6, 13, 9, 12, 15, 7, 14, 10, 8, 11)]
    vecs = [inputs.uniform(n, 900 + i) for i, n in enumerate(lengths)]
    check(env, lengths, vecs, run_batched(env, lengths, vecs, -1, graph=True), -1)


def test_every_large_split(env, monkeypatch):
    from paper_0811_2535_gb300 import inputs
    lengths = [1 << 13, 1 << 14, 1 << 15, 1 << 16]
    vecs = [inputs.uniform(n, 1200 + i) for i, n in enumerate(lengths)]
    for lr in range(3, 11):
        monkeypatch.setenv("MOA_BATCH_LOG2R", str(lr))
        check(env, lengths, vecs, run_batched(env, lengths, vecs, -1), -1)


def test_uneven_workload_full(env):
    """4096 transforms, lengths 2^k with k ~ U{6..16} (seed 2), N(0,1) data."""
    from paper_0811_2535_gb300 import inputs
    lengths, vecs = inputs.uneven_batch(4096, inputs.SEED_UNEVEN)
    lengths = [int(n) for n in lengths]
    check(env, lengths, vecs, run_batched(env, lengths, vecs, -1), -1)


def test_wait_timeout_is_reported_and_contained(env, monkeypatch):
    """Failure detection without a GPU fault: with MOA_FAULT_WAIT=1 at plan
    time every row tile of a large transform waits for a column-tile count
    that nothing reaches, with a short poll limit.  The launch completes, the
    status word reads MOA_ERR_TIMEOUT, the transforms that need no wait (the
    small ones) are still right, and the next plan on the same context runs
    correctly."""
    torch, moafft, _ = env
    from paper_0811_2535_gb300 import inputs
    lengths = [1 << 13, 64, 1 << 16, 256, 1 << 14, 4096, 128]
    vecs = [inputs.uniform(n, 1300 + i) for i, n in enumerate(lengths)]
    x = torch.from_numpy(np.concatenate(vecs)).cuda()
    monkeypatch.setenv("MOA_FAULT_WAIT", "1")
    plan = moafft.BatchedPlan(lengths, -1)
    monkeypatch.delenv("MOA_FAULT_WAIT")
    out = torch.zeros_like(x)
    plan.exec(x, out)
    torch.cuda.synchronize()
    assert plan.status() == moafft.MOA_ERR_TIMEOUT
    assert plan.status() == 0          # reading the status clears it
    offs = plan.offsets()
    plan.destroy()
    y = out.cpu().numpy()
    small = [i for i, n in enumerate(lengths) if n <= 4096]
    check(env, [lengths[i] for i in small], [vecs[i] for i in small],
          [y[offs[i]:offs[i] + lengths[i]] for i in small], -1)
    check(env, lengths, vecs, run_batched(env, lengths, vecs, -1), -1)
