"""The allocation-free entry point moa_fft_exec_noalloc (GPU).

It exists for callers that may not allocate device memory (their memory is
owned by a custom allocator, or their code path must never enter the CUDA
allocator); it keeps its scratch and twiddle tables in static device arrays.
This file is collected last so that a run stopping at the first failure has
already run every other test; it passes alone in a fresh process too.

Checks, through the C ABI: the output equals the planned transform's
(moa_fft_exec) within the parity tolerance, on two calls in a row; device
memory in use does not change across calls after the first; sizes beyond
the 2^20-point static scratch are rejected."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 2e-6
MOA_ERR_INVALID_SIZE, MOA_ERR_UNSUPPORTED = 2, 3


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0811_2535_gb300 import build, moafft
    build.build()
    return torch, moafft


def rel(a, b):
    a = np.asarray(a, np.complex128).reshape(-1)
    b = np.asarray(b, np.complex128).reshape(-1)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def noalloc(moafft, torch, x, out, sign):
    stream = torch.cuda.current_stream().cuda_stream
    return moafft.lib().moa_fft_exec_noalloc(x.data_ptr(), out.data_ptr(), x.numel(), sign, stream)


@pytest.mark.parametrize("t", [1, 10, 13, 16, 20])
@pytest.mark.parametrize("sign", [-1, 1])
def test_noalloc_matches_planned_transform_twice(env, t, sign):
    torch, moafft = env
    from paper_0811_2535_gb300 import inputs
    n = 1 << t
    x = torch.from_numpy(inputs.uniform(n, 7000 + t)).cuda()
    plan = moafft.Plan([n], 1, sign)
    ref = plan.exec(x).cpu().numpy()
    plan.destroy()
    for _ in range(2):
        out = torch.full_like(x, complex(float("nan"), 0.0))
        assert noalloc(moafft, torch, x, out, sign) == 0
        torch.cuda.synchronize()
        assert rel(out.cpu().numpy(), ref) <= TOL


def test_noalloc_in_place_and_memory_steady(env):
    torch, moafft = env
    from paper_0811_2535_gb300 import inputs
    n = 1 << 20
    x0 = inputs.uniform(n, 7100)
    x = torch.from_numpy(x0).cuda()
    out = torch.empty_like(x)
    assert noalloc(moafft, torch, x, out, -1) == 0          # first call: set-up on this device
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert noalloc(moafft, torch, x, out, -1) == 0
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    y = x.clone()
    assert noalloc(moafft, torch, y, y, -1) == 0            # in place
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), out.cpu().numpy()) <= TOL


def test_noalloc_rejects_sizes(env):
    torch, moafft = env
    L = moafft.lib()
    big = torch.empty(1 << 21, dtype=torch.complex64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert L.moa_fft_exec_noalloc(big.data_ptr(), big.data_ptr(), 1 << 21, -1, s) == MOA_ERR_UNSUPPORTED
    assert L.moa_fft_exec_noalloc(big.data_ptr(), big.data_ptr(), 3, -1, s) == MOA_ERR_INVALID_SIZE
    assert L.moa_fft_exec_noalloc(big.data_ptr(), big.data_ptr(), 1, -1, s) == MOA_ERR_INVALID_SIZE
    assert L.moa_fft_exec_noalloc(None, big.data_ptr(), 1024, -1, s) == 1
    assert L.moa_fft_exec_noalloc(big.data_ptr(), big.data_ptr(), 1024, 0, s) == 1
