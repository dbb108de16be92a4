"""Reduced-precision path (GPU): radix-16 DFT blocks on FP16 / BF16 tensor
cores with hi/lo operand splitting and FP32 accumulation, against the FP64
oracle.  Bar: relative L2 error <= 1e-5 per transform (the compensated
tensor-core tolerance), on inputs with large sinusoids (amplitude 10)."""
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


@pytest.mark.parametrize("dtype", [MOA_C64_TC_FP16, MOA_C64_TC_BF16])
@pytest.mark.parametrize("n", [256, 4096])
@pytest.mark.parametrize("sign", [-1, 1])
def test_tc_matches_oracle(env, dtype, n, sign):
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    batch = 48
    x = inputs.sinusoids(batch, n, 3000 + n + dtype)
    plan = moafft.Plan([n], batch, sign, dtype)
    assert plan.pass_info(0)["kernel"].startswith("tc_row_kernel")
    y = plan.exec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == 0
    plan.destroy()
    ref = oracle.fft_radix2(x.astype(np.complex128), sign)
    err = per_row_err(y, ref)
    assert err.max() <= TOL_TC, (dtype, n, err.max())


@pytest.mark.parametrize("dtype", [MOA_C64_TC_FP16, MOA_C64_TC_BF16])
def test_tc_uniform_and_tiny_and_huge_scales(env, dtype):
    """Power-of-two tile scaling keeps FP16 in range: inputs of very
    different magnitudes give the same relative accuracy."""
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    n, batch = 4096, 8
    base = inputs.uniform((batch, n), 31)
    plan = moafft.Plan([n], batch, -1, dtype)
    for scale in (1.0, 2.0 ** -20, 2.0 ** 20):
        x = (base * np.float32(scale)).astype(np.complex64)
        y = plan.exec(torch.from_numpy(x).cuda()).cpu().numpy()
        ref = oracle.fft_radix2(x.astype(np.complex128), -1)
        assert per_row_err(y, ref).max() <= TOL_TC, scale
    plan.destroy()


@pytest.mark.parametrize("dtype", [MOA_C64_TC_FP16, MOA_C64_TC_BF16])
def test_tc_precision_workload_sampled(env, dtype):
    """16384 x 4096, U[-1,1) noise plus 5 sinusoids of amplitude 10 per
    row (seed 3);
    sampled rows against the oracle."""
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    n, batch = 4096, 16384
    x = inputs.sinusoids(batch, n, inputs.SEED_PRECISION)
    plan = moafft.Plan([n], batch, -1, dtype)
    y = plan.exec(torch.from_numpy(x).cuda()).cpu().numpy()
    plan.destroy()
    rows = np.random.default_rng(5).choice(batch, 64, replace=False)
    ref = oracle.fft_radix2(x[rows].astype(np.complex128), -1)
    err = per_row_err(y[rows], ref)
    assert err.max() <= TOL_TC, err.max()
