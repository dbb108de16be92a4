"""The allocation-free entry points moa_fft_exec_noalloc and
moa_fft_noalloc_status (GPU).

They exist for callers that may not allocate device memory (their memory is
owned by a custom allocator, or their code path must never enter the CUDA
allocator); the transform keeps its scratch and twiddle tables in static
device arrays.  This file is collected last so that a run stopping at the
first failure has already run every other test; it passes alone in a fresh
process too.

Checks, through the C ABI: the output equals the FP64 oracle's within the
parity tolerance (rel-L2 <= 2e-6), on two calls in a row, for one-tile,
lifted and pipelined sizes, both signs, in place too; the status word reads
MOA_OK after each call; device memory in use does not change across calls
after the first; a wait that gives up (the short-wait fault injection, no
GPU fault) is reported through moa_fft_noalloc_status and the next call is
right again; sizes beyond the 2^20-point static scratch are rejected."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 2e-6
MOA_OK, MOA_ERR_INVALID_ARG, MOA_ERR_INVALID_SIZE, MOA_ERR_UNSUPPORTED, MOA_ERR_TIMEOUT = 0, 1, 2, 3, 6


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0811_2535_gb300 import build, moafft
    import oracle
    build.build()
    oracle.build()
    return torch, moafft, oracle


def rel(a, b):
    a = np.asarray(a, np.complex128).reshape(-1)
    b = np.asarray(b, np.complex128).reshape(-1)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def stream_of(torch):
    return torch.cuda.current_stream().cuda_stream


def noalloc(moafft, torch, x, out, sign):
    return moafft.lib().moa_fft_exec_noalloc(x.data_ptr(), out.data_ptr(), x.numel(), sign, stream_of(torch))


def status(moafft, torch):
    return moafft.lib().moa_fft_noalloc_status(stream_of(torch))


@pytest.mark.parametrize("t", [1, 10, 13, 16, 19, 20])
@pytest.mark.parametrize("sign", [-1, 1])
def test_noalloc_matches_oracle_twice(env, t, sign):
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    n = 1 << t
    x0 = inputs.uniform(n, 7000 + t)
    ref = oracle.fft_radix2(x0.astype(np.complex128), sign)
    x = torch.from_numpy(x0).cuda()
    for _ in range(2):
        out = torch.full_like(x, complex(float("nan"), 0.0))
        assert noalloc(moafft, torch, x, out, sign) == MOA_OK
        assert status(moafft, torch) == MOA_OK
        assert rel(out.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("t", [10, 19, 20])
def test_noalloc_in_place(env, t):
    """One row pass (2^10), the odd split with a pipelined row pass (2^19 =
    2^9 x 2^10) and the two pipelined passes (2^20), each with in == out."""
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    n = 1 << t
    x0 = inputs.uniform(n, 7100 + t)
    ref = oracle.fft_radix2(x0.astype(np.complex128), -1)
    y = torch.from_numpy(x0).cuda()
    assert noalloc(moafft, torch, y, y, -1) == MOA_OK
    assert status(moafft, torch) == MOA_OK
    assert rel(y.cpu().numpy(), ref) <= TOL


def test_noalloc_memory_steady(env):
    torch, moafft, _ = env
    from paper_0811_2535_gb300 import inputs
    n = 1 << 20
    x = torch.from_numpy(inputs.uniform(n, 7200)).cuda()
    out = torch.empty_like(x)
    assert noalloc(moafft, torch, x, out, -1) == MOA_OK      # first call: set-up on this device
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert noalloc(moafft, torch, x, out, -1) == MOA_OK
    assert status(moafft, torch) == MOA_OK
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before


def test_noalloc_wait_timeout_is_reported(env, monkeypatch):
    """Failure detection without a GPU fault: with MOA_FAULT_WAIT=1 at call
    time the pipelined kernels of a 2^20 transform give up on the first tile
    load that has not landed at its first test; each block then waits for its
    loads in flight and returns.  The status word reads MOA_ERR_TIMEOUT once
    and is then clear, and the next call is right."""
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    n = 1 << 20
    x0 = inputs.uniform(n, 7300)
    x = torch.from_numpy(x0).cuda()
    out = torch.empty_like(x)
    assert noalloc(moafft, torch, x, out, -1) == MOA_OK      # set-up before the fault knob
    assert status(moafft, torch) == MOA_OK
    monkeypatch.setenv("MOA_FAULT_WAIT", "1")
    assert noalloc(moafft, torch, x, out, -1) == MOA_OK
    monkeypatch.delenv("MOA_FAULT_WAIT")
    assert status(moafft, torch) == MOA_ERR_TIMEOUT
    assert status(moafft, torch) == MOA_OK                   # reading clears it
    assert noalloc(moafft, torch, x, out, -1) == MOA_OK
    assert status(moafft, torch) == MOA_OK
    assert rel(out.cpu().numpy(), oracle.fft_radix2(x0.astype(np.complex128), -1)) <= TOL


def test_noalloc_rejects_sizes(env):
    torch, moafft, _ = env
    L = moafft.lib()
    big = torch.empty(1 << 21, dtype=torch.complex64, device="cuda")
    s = stream_of(torch)
    assert L.moa_fft_exec_noalloc(big.data_ptr(), big.data_ptr(), 1 << 21, -1, s) == MOA_ERR_UNSUPPORTED
    assert L.moa_fft_exec_noalloc(big.data_ptr(), big.data_ptr(), 3, -1, s) == MOA_ERR_INVALID_SIZE
    assert L.moa_fft_exec_noalloc(big.data_ptr(), big.data_ptr(), 1, -1, s) == MOA_ERR_INVALID_SIZE
    assert L.moa_fft_exec_noalloc(None, big.data_ptr(), 1024, -1, s) == MOA_ERR_INVALID_ARG
    assert L.moa_fft_exec_noalloc(big.data_ptr(), big.data_ptr(), 1024, 0, s) == MOA_ERR_INVALID_ARG
