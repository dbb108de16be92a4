"""Radix schedules and the warp-shuffle row kernel (GPU), against the FP64
oracle at the parity tolerance (rel-L2 <= 2e-6 per transform).

Sec. 4.8: every breakpoint of the lifting gives the same transform, so each
schedule of the in-register stages must match the oracle on its own:
  MOA_SCHED=1  radix 16 stages with the small radix last (L = 9, 10, 11),
  MOA_SCHED=2  radix-8 stages (L = 7..12),
  MOA_SCHED=3  the warp-shuffle row kernel (natural-order rows of 128, 256,
               512 points: radix 16 in registers, then the butterflies that
               cross lanes by shfl.xor, no shared-memory exchange).
The plan is asked for each schedule through MOA_SCHED with the autotuner off,
and the kernel names it reports show that the schedule was used.  The stage
tables of each schedule are checked entry by entry like the default ones."""
import numpy as np
import pytest

from test_gpu_twiddles import root64, ulps

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


@pytest.fixture
def sched(monkeypatch):
    monkeypatch.setenv("MOA_AUTOTUNE", "0")

    def set_sched(v, pipe=None):
        monkeypatch.setenv("MOA_SCHED", str(v))
        if pipe is not None:
            monkeypatch.setenv("MOA_PIPE", str(pipe))
    return set_sched


def rel(y, ref, batch):
    y = np.asarray(y, np.complex128).reshape(batch, -1)
    ref = np.asarray(ref, np.complex128).reshape(batch, -1)
    return np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)


def run(env, shape, batch, sign, x, inplace=False):
    torch, moafft, oracle = env
    plan = moafft.Plan(list(shape), batch, sign)
    names = [plan.pass_info(i)["kernel"] for i in range(plan.info()["passes"])]
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = plan.exec(xd, out=xd) if inplace else plan.exec(xd)
    y = out.cpu().numpy()
    assert plan.status() == 0
    plan.destroy()
    x64 = np.asarray(x, np.complex128).reshape((batch,) + tuple(shape))
    ref = oracle.fft_radix2(x64, sign) if len(shape) == 1 else oracle.fft_nd(x64, len(shape), sign)
    return rel(y, ref, batch), names


@pytest.mark.parametrize("v,L", [(1, 9), (1, 10), (1, 11), (2, 7), (2, 8), (2, 9), (2, 10), (2, 11), (2, 12)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_schedule_rows(env, sched, v, L, sign):
    """Natural-order rows, batch 37: several tiles and a ragged last one."""
    from paper_0811_2535_gb300 import inputs
    sched(v)
    n, batch = 1 << L, 37
    x = inputs.uniform((batch, n), 8000 + 10 * v + L)
    err, names = run(env, [n], batch, sign, x)
    assert names == [f"row_pass_kernel<{L},0,{v}>"]
    assert err.max() <= TOL, err.max()


@pytest.mark.parametrize("v,L,lr", [(1, 20, 10), (1, 19, 9), (2, 16, 8), (2, 21, 10), (2, 14, 7)])
def test_schedule_lifted_generic(env, sched, v, L, lr, monkeypatch):
    """The lifted 1-D transform on the generic kernels: the column pass with
    the four-step twiddle and the transposed row pass, both in schedule v."""
    from paper_0811_2535_gb300 import inputs
    sched(v, pipe=0)
    monkeypatch.setenv("MOA_SPLIT_LOG2R", str(lr))
    n, batch = 1 << L, 2
    x = inputs.uniform((batch, n), 8100 + 10 * v + L)
    err, names = run(env, [n], batch, -1, x)
    lc = L - lr
    want = [f"col_pass_kernel<{lr},1,{v}>" if (v == 2 and lr >= 7) or (v == 1 and 9 <= lr <= 11)
            else f"col_pass_kernel<{lr},1>",
            f"row_pass_kernel<{lc},1,{v}>" if (v == 2 and lc >= 7) or (v == 1 and 9 <= lc <= 11)
            else f"row_pass_kernel<{lc},1>"]
    assert names == want
    assert err.max() <= TOL, err.max()


@pytest.mark.parametrize("v", [1, 2])
@pytest.mark.parametrize("shape,batch", [((512, 128), 2), ((1024, 2048), 1), ((128, 4, 512), 1)])
def test_schedule_multi_d(env, sched, v, shape, batch):
    from paper_0811_2535_gb300 import inputs
    sched(v, pipe=0)
    x = inputs.uniform((batch,) + shape, 8200 + v + sum(shape))
    err, names = run(env, shape, batch, 1, x)
    assert any(f",{v}>" in nm for nm in names), names
    assert err.max() <= TOL, err.max()


@pytest.mark.parametrize("L", [7, 8, 9])
@pytest.mark.parametrize("batch", [1, 4, 37, 1000])
@pytest.mark.parametrize("sign", [-1, 1])
def test_warp_shuffle_rows(env, sched, L, batch, sign):
    """row_warp_kernel wherever its blocks are whole warps (32 threads or
    more); smaller blocks keep the shared-memory kernel."""
    from paper_0811_2535_gb300 import inputs
    sched(3)
    n = 1 << L
    x = inputs.uniform((batch, n), 8300 + L + batch)
    err, names = run(env, [n], batch, sign, x)
    T = n // 16
    lf = min(12 - L, (batch - 1).bit_length())
    assert names == ([f"row_warp_kernel<{L}>"] if (T << lf) % 32 == 0 else [f"row_pass_kernel<{L},0>"])
    assert err.max() <= TOL, err.max()


@pytest.mark.parametrize("shape,batch", [((512,), 64), ((256, 128), 3), ((4, 4, 256), 5)])
def test_warp_shuffle_in_place_and_multi_d(env, sched, shape, batch):
    """In place (each warp reads all of its rows before it writes them), and as
    the last-axis pass of multi-D arrays."""
    from paper_0811_2535_gb300 import inputs
    sched(3, pipe=0)
    x = inputs.uniform((batch,) + shape, 8400 + sum(shape) + batch)
    err, names = run(env, shape, batch, -1, x, inplace=True)
    assert names[0] == f"row_warp_kernel<{shape[-1].bit_length() - 1}>"
    assert err.max() <= TOL, err.max()


def schedule_radices(L, v):
    """Radix logs of schedule v, restated from its definition."""
    if v == 2:
        S = 1 if L <= 3 else (L + 2) // 3
        return [L] if L <= 3 else [(L % 3) if (s == 0 and L % 3) else 3 for s in range(S)]
    S = (L + 3) // 4
    return [(L % 4) if (s == S - 1 and L % 4) else 4 for s in range(S)]


def schedule_table(L, v):
    N = 1 << L
    if v == 3:   # rows k = 1, 2, 3, 4, 8, 12 of w_N^(u k), u < T, then w_T^u
        T = N // 16
        u = np.arange(T, dtype=np.int64)
        return np.concatenate([root64(u * k, N) for k in (1, 2, 3, 4, 8, 12)] + [root64(u, T)])
    rl = schedule_radices(L, v)
    assert sum(rl) == L
    parts, K = [], 1
    for s in range(len(rl) - 1):
        R = 1 << rl[s]
        M1 = N // K // R
        u = np.arange(M1, dtype=np.int64)
        parts += [root64(u * k, M1 * R) for k in (1, 2, 3, 4, 8, 12)]
        K *= R
    return np.concatenate(parts)


@pytest.mark.parametrize("v,L", [(1, 9), (1, 10), (1, 11), (2, 7), (2, 9), (2, 12), (3, 7), (3, 8), (3, 9)])
def test_schedule_tables_correctly_rounded(env, sched, v, L):
    _, moafft, _ = env
    sched(v)
    plan = moafft.Plan([1 << L], 64, -1)
    t = plan.table(2 + v, L)
    plan.destroy()
    ref = schedule_table(L, v)
    assert t.shape == ref.shape
    assert ulps(t, ref).max() <= 1


@pytest.mark.parametrize("v,shape,batch", [(1, (2048,), 100), (2, (4096,), 50), (3, (256,), 300), (3, (512,), 64),
                                           (2, (1 << 18,), 3)])
def test_schedule_adjoint_and_round_trip(env, sched, v, shape, batch):
    """The adjoint (opposite-sign, unnormalised) transform on the same plan,
    against the oracle's +1 transform, and exec then adjoint = n * x."""
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    sched(v, pipe=0)
    x = inputs.uniform((batch,) + shape, 8500 + v + batch)
    plan = moafft.Plan(list(shape), batch, -1)
    xd = torch.from_numpy(x).cuda()
    a = plan.exec_adjoint(xd).cpu().numpy()
    y = plan.exec(xd)
    z = plan.exec_adjoint(y).cpu().numpy()
    assert plan.status() == 0
    plan.destroy()
    x64 = x.astype(np.complex128).reshape((batch,) + shape)
    assert rel(a, oracle.fft_radix2(x64, 1), batch).max() <= TOL
    n = int(np.prod(shape))
    assert rel(z / n, x64, batch).max() <= 2 * TOL


@pytest.mark.parametrize("v,shape,batch", [(3, (512,), 65), (3, (128,), 40), (1, (1024,), 9), (2, (4096,), 3)])
def test_schedule_eight_byte_aligned(env, sched, v, shape, batch):
    """Buffers one complex64 past a 16-byte boundary (the ABI asks for 8-byte
    alignment only), out of place and in place."""
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    sched(v)
    n = int(np.prod(shape)) * batch
    x = inputs.uniform((batch,) + shape, 8600 + v + batch)
    bin_ = torch.empty(n + 1, dtype=torch.complex64, device="cuda")
    bout = torch.empty(n + 1, dtype=torch.complex64, device="cuda")
    xin, yout = bin_[1:], bout[1:]
    assert xin.data_ptr() % 16 == 8 and yout.data_ptr() % 16 == 8
    xin.copy_(torch.from_numpy(x.reshape(-1)))
    plan = moafft.Plan(list(shape), batch, -1)
    plan.exec(xin, out=yout)
    plan.exec(xin, out=xin)
    assert plan.status() == 0
    plan.destroy()
    ref = oracle.fft_radix2(x.astype(np.complex128).reshape((batch,) + shape), -1)
    assert rel(yout.cpu().numpy(), ref, batch).max() <= TOL
    assert rel(xin.cpu().numpy(), ref, batch).max() <= TOL


@pytest.mark.parametrize("v,shape,batch", [(3, (256,), 1000), (1, (1 << 19,), 2)])
def test_schedule_cuda_graph(env, sched, v, shape, batch):
    """Execs in schedule v captured in a CUDA graph and replayed twice give
    the bits of the same execs run directly."""
    torch, _, _ = env
    from paper_0811_2535_gb300 import inputs, moafft
    sched(v, pipe=0)
    x = torch.from_numpy(inputs.uniform((batch,) + shape, 8700 + v)).cuda()
    plan = moafft.Plan(list(shape), batch, -1)
    y = torch.empty_like(x)
    plan.exec(x, y)
    torch.cuda.synchronize()
    ref = y.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.exec(x, y)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.exec(x, y)
    for _ in range(2):
        y.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(y, ref)
    assert plan.status() == 0
    plan.destroy()


@pytest.mark.parametrize("v,L", [(2, 12), (1, 11), (3, 9)])
def test_schedule_full_size_sampled(env, sched, v, L):
    """2^24 points of rows (the size of the benchmark's transforms) in schedule
    v: 64 sampled rows against the oracle one by one."""
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    sched(v)
    n, batch = 1 << L, (1 << 24) >> L
    x = inputs.uniform((batch, n), 8800 + L)
    plan = moafft.Plan([n], batch, -1)
    y = plan.exec(torch.from_numpy(x).cuda()).cpu().numpy().reshape(batch, n)
    assert plan.status() == 0
    plan.destroy()
    rows = np.random.default_rng(L).choice(batch, 64, replace=False)
    ref = oracle.fft_radix2(x[rows].astype(np.complex128), -1)
    assert rel(y[rows], ref, 64).max() <= TOL
