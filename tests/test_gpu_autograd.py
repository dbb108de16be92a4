"""Differentiation through the transform (GPU).

loss = sum |H * F(x)|^2 with F the forward transform wrapped in
MoaFFTFunction, whose backward pass is the adjoint kernel (the
opposite-sign unnormalised transform on the same plan).  In PyTorch's
convention for complex inputs the gradient is dL/dRe + i dL/dIm, which for
this quadratic loss equals 2 F^H (|H|^2 * F x).

Checks: FP64 central finite differences of the loss evaluated with the
oracle (exact up to rounding, L is quadratic) at n = 2^8; the closed form
evaluated with the oracle at n = 2^8 and on sampled rows of the full-size
batch 256 x 2^18 workload."""
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


def gpu_grad(env, H, x, n, batch):
    torch, moafft, _ = env
    plan = moafft.Plan([n], batch, -1)
    xd = torch.from_numpy(x.reshape(batch, n)).cuda().requires_grad_(True)
    Hd = torch.from_numpy(H).cuda()
    y = moafft.fft_autograd(xd, plan)
    loss = (Hd * y).abs().pow(2).sum()
    loss.backward()
    g = xd.grad.detach().cpu().numpy()
    assert plan.status() == 0
    plan.destroy()
    return float(loss.item()), g


def oracle_loss(oracle, H, x):
    y = oracle.fft_radix2(x.astype(np.complex128), -1)
    return float(np.sum(np.abs(H.astype(np.complex128) * y) ** 2))


def oracle_grad(oracle, H, x):
    x = x.astype(np.complex128)
    h2 = np.abs(H.astype(np.complex128)) ** 2
    y = oracle.fft_radix2(x, -1)
    return 2.0 * oracle.fft_radix2(h2 * y, +1)       # F^H = sign +1 transform


def test_gradient_matches_fp64_finite_differences(env):
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    n = 1 << 8
    H, x = inputs.spectral_filter(n, 1, inputs.SEED_GRADIENT)
    x = x.reshape(n)
    loss, g = gpu_grad(env, H, x, n, 1)
    assert abs(loss - oracle_loss(oracle, H, x)) / oracle_loss(oracle, H, x) < 1e-5
    x64 = x.astype(np.complex128)
    h = 1e-3
    fd = np.empty(n, np.complex128)
    for j in range(n):
        parts = []
        for unit in (1.0, 1j):
            xp = x64.copy()
            xm = x64.copy()
            xp[j] += h * unit
            xm[j] -= h * unit
            parts.append((oracle_loss(oracle, H, xp) - oracle_loss(oracle, H, xm)) / (2 * h))
        fd[j] = parts[0] + 1j * parts[1]
    g = g.reshape(n).astype(np.complex128)
    assert np.linalg.norm(g - fd) / np.linalg.norm(fd) < 1e-5
    # and the closed form through the oracle's adjoint
    ref = oracle_grad(oracle, H, x)
    assert np.linalg.norm(fd - ref) / np.linalg.norm(ref) < 1e-9     # pins the closed form itself
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) <= TOL


def test_gradient_full_size_batch_sampled(env):
    """batch 256 x n = 2^18 (seed 4): gradient rows checked against the
    oracle's closed form on a sample of rows."""
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    n, batch = 1 << 18, 256
    H, x = inputs.spectral_filter(n, batch, inputs.SEED_GRADIENT)
    _, g = gpu_grad(env, H, x, n, batch)
    g = g.reshape(batch, n)
    for b in (0, 1, 127, 255):
        ref = oracle_grad(oracle, H, x[b])
        err = np.linalg.norm(g[b].astype(np.complex128) - ref) / np.linalg.norm(ref)
        assert err <= TOL, (b, err)


def test_vector_jacobian_product_is_adjoint(env):
    """For y = F x and any cotangent v, the backward pass returns F^H v
    (the map is linear, nothing is saved for backward)."""
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    n = 1 << 12
    x = inputs.uniform(n, 21)
    v = inputs.uniform(n, 22)
    plan = moafft.Plan([n], 1, -1)
    xd = torch.from_numpy(x).cuda().requires_grad_(True)
    y = moafft.fft_autograd(xd, plan)
    y.backward(torch.from_numpy(v).cuda())
    ref = oracle.fft_radix2(v.astype(np.complex128), +1)
    got = xd.grad.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL
