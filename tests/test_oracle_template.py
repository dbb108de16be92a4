"""Pins of the all-processor templates (Sec. 6.3, Fig. 6.4; Eq. B.6 in
parallel) that give the CPU comparison point (CPU only).

The templates run the butterflies of the sequential plans with the same
weights in the same stage order, only spread over threads, so their results
must equal the sequential oracle bit for bit; they are also checked against
the DFT definition and numpy.fft directly, so that a mistake shared with the
sequential plan would still show.
"""
import numpy as np
import pytest


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rand_c(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)


def test_template_threads(oracle):
    assert oracle.template_threads() >= 1


@pytest.mark.parametrize("t", range(1, 13))
@pytest.mark.parametrize("sign", [-1, 1])
def test_template_partitioned_every_split(oracle, t, sign):
    n = 1 << t
    x = rand_c(n, 900 + t)
    ref = oracle.dft_naive(x, sign) if n <= 256 else np.fft.fft(x) if sign < 0 else np.fft.ifft(x) * n
    checked = 0
    m = 1
    while m <= n // m:
        lo, hi = int(np.log2(m)) + 1, int(np.log2(n // m)) + 1
        for bp in range(lo, hi + 1):
            y = oracle.template_partitioned(x, m, bp, sign)
            np.testing.assert_array_equal(y, oracle.fft_partitioned(x, m, bp, sign))
            assert rel_l2(y, ref) < 1e-13, (m, bp)
            checked += 1
        with pytest.raises(ValueError):
            oracle.template_partitioned(x, m, lo - 1, sign)
        with pytest.raises(ValueError):
            oracle.template_partitioned(x, m, hi + 1, sign)
        m *= 2
    assert checked >= 1


def test_template_partitioned_rejects_bad_arguments(oracle):
    x = rand_c(64, 1)
    for m, bp in ((3, 3), (0, 1), (16, 5)):       # not a power of two; zero; m > psize
        with pytest.raises(ValueError):
            oracle.template_partitioned(x, m, bp, -1)
    with pytest.raises(ValueError):
        oracle.template_partitioned(x, 4, 3, 0)    # sign
    with pytest.raises(ValueError):
        oracle.template_partitioned(rand_c(48, 1), 4, 3, -1)


def test_template_partitioned_large_equals_sequential(oracle):
    """2^20 points on up to 16 processors with the default breakpoint
    log2(psize) + 1: the same butterflies as the sequential Fig. 2.1 loop."""
    t = 20
    x = rand_c(1 << t, 31)
    m = 1
    while m * 2 <= min(16, oracle.template_threads() * 2):
        m *= 2
    y = oracle.template_partitioned(x, m, t - int(np.log2(m)) + 1, -1)
    np.testing.assert_array_equal(y, oracle.fft_radix2(x, -1))
    assert rel_l2(y, np.fft.fft(x)) < 1e-12


@pytest.mark.parametrize("shape,dims", [((8,), 1), ((3, 4, 16), 2), ((2, 8, 4, 32), 3), ((256,), 1),
                                        ((2, 2), 2)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_template_nd_equals_sequential_and_numpy(oracle, shape, dims, sign):
    x = rand_c(shape, 77)
    y = oracle.template_nd(x, dims, sign)
    np.testing.assert_array_equal(y, oracle.fft_nd(x, dims, sign))
    axes = tuple(range(len(shape) - dims, len(shape)))
    ref = np.fft.fftn(x, axes=axes) if sign < 0 else np.fft.ifftn(x, axes=axes) * np.prod([shape[a] for a in axes])
    assert rel_l2(y, ref) < 1e-13


def test_template_nd_inplace_and_bad_shapes(oracle):
    x = rand_c((16, 32), 5)
    ref = oracle.fft_nd(x, 2, -1)
    oracle.template_nd(x, 2, -1, inplace=True)
    np.testing.assert_array_equal(x, ref)
    with pytest.raises(ValueError):
        oracle.template_nd(rand_c((6, 8), 1), 2, -1)
    with pytest.raises(ValueError):
        oracle.template_nd(rand_c((8, 8), 1).astype(np.complex64), 2, -1, inplace=True)
