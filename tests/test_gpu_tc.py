"""Reduced-precision path (GPU): radix-16 DFT blocks on FP16 / BF16 tensor
cores with hi/lo operand splitting and FP32 accumulation, against the FP64
oracle.  Bar: relative L2 error <= 1e-5 per transform (the compensated
tensor-core tolerance), on inputs with large sinusoids (amplitude 10).
Both kernels: tcgen05 (default) and mma.sync (MOA_TC_KERNEL=sync)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_TC = 1e-5
MOA_C64_TC_FP16, MOA_C64_TC_BF16 = 1, 2


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


def per_row_err(y, ref):
    y = np.asarray(y, np.complex128).reshape(ref.shape)
    return np.linalg.norm(y - ref, axis=-1) / np.linalg.norm(ref, axis=-1)


KERNELS = [("", "tc_umma_kernel"), ("sync", "tc_row_kernel")]


@pytest.mark.parametrize("kernel", KERNELS, ids=["tcgen05", "mma_sync"])
@pytest.mark.parametrize("dtype", [MOA_C64_TC_FP16, MOA_C64_TC_BF16])
@pytest.mark.parametrize("n,batch", [(256, 48), (4096, 48), (256, 37), (256, 1), (4096, 1)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_tc_matches_oracle(env, kernel, dtype, n, batch, sign, monkeypatch):
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    monkeypatch.setenv("MOA_TC_KERNEL", kernel[0])
    x = inputs.sinusoids(batch, n, 3000 + n + dtype + batch)
    plan = moafft.Plan([n], batch, sign, dtype)
    assert plan.pass_info(0)["kernel"].startswith(kernel[1])
    y = plan.exec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == 0
    plan.destroy()
    ref = oracle.fft_radix2(x.astype(np.complex128), sign)
    err = per_row_err(y, ref)
    assert err.max() <= TOL_TC, (dtype, n, err.max())


@pytest.mark.parametrize("kernel", KERNELS, ids=["tcgen05", "mma_sync"])
@pytest.mark.parametrize("dtype", [MOA_C64_TC_FP16, MOA_C64_TC_BF16])
def test_tc_uniform_and_tiny_and_huge_scales(env, kernel, dtype, monkeypatch):
    """Power-of-two tile scaling keeps FP16 in range: inputs of very
    different magnitudes give the same relative accuracy."""
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    monkeypatch.setenv("MOA_TC_KERNEL", kernel[0])
    n, batch = 4096, 8
    base = inputs.uniform((batch, n), 31)
    plan = moafft.Plan([n], batch, -1, dtype)
    for scale in (1.0, 2.0 ** -20, 2.0 ** 20):
        x = (base * np.float32(scale)).astype(np.complex64)
        y = plan.exec(torch.from_numpy(x).cuda()).cpu().numpy()
        ref = oracle.fft_radix2(x.astype(np.complex128), -1)
        assert per_row_err(y, ref).max() <= TOL_TC, scale
    plan.destroy()


@pytest.mark.parametrize("kernel", KERNELS, ids=["tcgen05", "mma_sync"])
@pytest.mark.parametrize("dtype", [MOA_C64_TC_FP16, MOA_C64_TC_BF16])
def test_tc_precision_workload_sampled(env, kernel, dtype, monkeypatch):
    """16384 x 4096, U[-1,1) noise plus 5 sinusoids of amplitude 10 per
    row (seed 3);
    sampled rows against the oracle."""
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    monkeypatch.setenv("MOA_TC_KERNEL", kernel[0])
    n, batch = 4096, 16384
    x = inputs.sinusoids(batch, n, inputs.SEED_PRECISION)
    plan = moafft.Plan([n], batch, -1, dtype)
    y = plan.exec(torch.from_numpy(x).cuda()).cpu().numpy()
    plan.destroy()
    rows = np.random.default_rng(5).choice(batch, 64, replace=False)
    ref = oracle.fft_radix2(x[rows].astype(np.complex128), -1)
    err = per_row_err(y[rows], ref)
    assert err.max() <= TOL_TC, err.max()


def test_tc_in_place(env):
    """in == out: every block of 4096 points is read before it is written."""
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    for n, batch in ((4096, 300), (256, 333)):
        x = inputs.sinusoids(batch, n, 77)
        plan = moafft.Plan([n], batch, -1, MOA_C64_TC_FP16)
        xd = torch.from_numpy(x).cuda()
        y = plan.exec(xd, out=xd).cpu().numpy()
        assert plan.status() == 0
        plan.destroy()
        ref = oracle.fft_radix2(x.astype(np.complex128), -1)
        assert per_row_err(y, ref).max() <= TOL_TC
