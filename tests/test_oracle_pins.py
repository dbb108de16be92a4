"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks the oracle against what the paper or the mathematics fixes:
brute force (the DFT definition at small n), a library routine for the
special case it implements (numpy.fft), closed forms, invariants (Parseval,
linearity, round trip, adjoint), the paper's own correctness claim that
every breakpoint of the partitioned plan gives the same result (Sec. 4.8),
split invariance of the dimension-lifting form, Omega separability
(Appendix B) and the worked psi example of Appendix A.1.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rand_c(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, n) + 1j * rng.uniform(-1, 1, n)


# -- the definition itself --------------------------------------------------

def test_naive_dft_textbook_4_point(oracle):
    # The 4-point DFT matrix with exp(-2 pi i/4) = -i: rows (1,1,1,1),
    # (1,-i,-1,i), (1,-1,1,-1), (1,i,-1,-i); the +1 sign conjugates it.
    F = np.array([[1, 1, 1, 1], [1, -1j, -1, 1j], [1, -1, 1, -1], [1, 1j, -1, -1j]])
    x = np.array([1 + 2j, -0.5 + 0.25j, 3 - 1j, 0.125 + 0j])
    np.testing.assert_allclose(oracle.dft_naive(x, -1), F @ x, rtol=0, atol=1e-14)
    np.testing.assert_allclose(oracle.dft_naive(x, +1), F.conj() @ x, rtol=0, atol=1e-14)
    # n = 2: [a + b, a - b] for either sign
    np.testing.assert_allclose(oracle.dft_naive([3 + 1j, 1 - 2j], -1), [4 - 1j, 2 + 3j], atol=1e-15)


@pytest.mark.parametrize("t", range(1, 9))
def test_naive_dft_matches_numpy(oracle, t):
    n = 1 << t
    x = rand_c(n, 100 + t)
    assert rel_l2(oracle.dft_naive(x, -1), np.fft.fft(x)) < 1e-13
    assert rel_l2(oracle.dft_naive(x, +1), n * np.fft.ifft(x)) < 1e-13


# -- Fig. 2.1 / Sec. 3.6 radix-2 loop ----------------------------------------

@pytest.mark.parametrize("t", range(1, 9))
@pytest.mark.parametrize("sign", [-1, 1])
def test_radix2_equals_brute_force_dft(oracle, t, sign):
    n = 1 << t
    x = rand_c(n, 200 + t)
    assert rel_l2(oracle.fft_radix2(x, sign), oracle.dft_naive(x, sign)) < 1e-13


@pytest.mark.parametrize("t", [9, 12, 16, 20])
def test_radix2_matches_numpy_large(oracle, t):
    n = 1 << t
    x = rand_c(n, 300 + t)
    assert rel_l2(oracle.fft_radix2(x, -1), np.fft.fft(x)) < 1e-13
    assert rel_l2(oracle.fft_radix2(x, +1), n * np.fft.ifft(x)) < 1e-13


@pytest.mark.parametrize("t", [1, 2, 3, 5, 8, 11, 14, 17, 20])
@pytest.mark.parametrize("sign", [-1, 1])
def test_radix2_closed_forms(oracle, t, sign):
    n = 1 << t
    j = np.arange(n)
    k = np.arange(n)
    # delta at 0 -> all ones
    d = np.zeros(n, complex)
    d[0] = 1
    np.testing.assert_allclose(oracle.fft_radix2(d, sign), np.ones(n), atol=1e-12)
    # delta at j0 -> w_n^(j0 k), w_n = exp(sign 2 pi i / n)
    j0 = (5 * n) // 7 if n > 2 else 1
    d = np.zeros(n, complex)
    d[j0] = 1
    expect = np.exp(sign * 2j * np.pi * ((j0 * k) % n) / n)
    np.testing.assert_allclose(oracle.fft_radix2(d, sign), expect, atol=1e-12)
    # exp(-sign 2 pi i f j / n) -> n at bin f, 0 elsewhere
    f = (3 * n) // 5 if n > 2 else 1
    x = np.exp(-sign * 2j * np.pi * ((f * j) % n) / n)
    y = oracle.fft_radix2(x, sign)
    onehot = np.zeros(n, complex)
    onehot[f] = n
    assert np.max(np.abs(y - onehot)) < 1e-12 * n * max(t, 1)
    # cos(2 pi f j / n) -> n/2 at bins f and n - f (n at bin f when f = n - f)
    x = np.cos(2 * np.pi * ((f * j) % n) / n)
    y = oracle.fft_radix2(x, sign)
    expect = np.zeros(n, complex)
    expect[f] += n / 2
    expect[(n - f) % n] += n / 2
    assert np.max(np.abs(y - expect)) < 1e-12 * n * max(t, 1)
    # constant -> n at bin 0
    y = oracle.fft_radix2(np.ones(n), sign)
    expect = np.zeros(n, complex)
    expect[0] = n
    assert np.max(np.abs(y - expect)) < 1e-12 * n


@pytest.mark.parametrize("t", [4, 10, 16])
def test_radix2_invariants(oracle, t):
    n = 1 << t
    x = rand_c(n, 400 + t)
    z = rand_c(n, 500 + t)
    X = oracle.fft_radix2(x, -1)
    # Parseval
    assert abs(np.vdot(X, X).real - n * np.vdot(x, x).real) / (n * np.vdot(x, x).real) < 1e-12
    # linearity
    a, b = 0.75 - 1.5j, -2.0 + 0.5j
    lhs = oracle.fft_radix2(a * x + b * z, -1)
    rhs = a * X + b * oracle.fft_radix2(z, -1)
    assert rel_l2(lhs, rhs) < 1e-13
    # round trip F_{+} F_{-} x = n x
    assert rel_l2(oracle.fft_radix2(X, +1) / n, x) < 1e-13
    # adjoint identity <F x, z> = <x, F^H z>, F^H = opposite sign transform
    lhs = np.vdot(z, X)
    rhs = np.vdot(oracle.fft_radix2(z, +1), x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_radix2_rejects_bad_sizes(oracle):
    for bad in (1, 3, 6, 12):
        with pytest.raises(ValueError):
            oracle.fft_radix2(np.ones(bad, complex), -1)


# -- Sec. 4.8: every breakpoint of the Fig. 4.9 plan gives the same result ---

@pytest.mark.parametrize("t", range(1, 11))
@pytest.mark.parametrize("sign", [-1, 1])
def test_partitioned_plan_breakpoint_invariance(oracle, t, sign):
    n = 1 << t
    x = rand_c(n, 600 + t)
    ref = oracle.dft_naive(x, sign) if n <= 256 else oracle.fft_radix2(x, sign)
    checked = 0
    m = 1
    while m <= n // m:
        psize = n // m
        lo, hi = int(np.log2(m)) + 1, int(np.log2(psize)) + 1
        for bp in range(lo, hi + 1):
            assert rel_l2(oracle.fft_partitioned(x, m, bp, sign), ref) < 1e-13, (m, bp)
            checked += 1
        with pytest.raises(ValueError):
            oracle.fft_partitioned(x, m, lo - 1, sign)
        with pytest.raises(ValueError):
            oracle.fft_partitioned(x, m, hi + 1, sign)
        m *= 2
    assert checked >= 1


# -- dimension lifting n = r*c ----------------------------------------------

@pytest.mark.parametrize("t", range(1, 13))
@pytest.mark.parametrize("sign", [-1, 1])
def test_four_step_every_split(oracle, t, sign):
    n = 1 << t
    x = rand_c(n, 700 + t)
    ref = oracle.dft_naive(x, sign) if n <= 256 else np.fft.fft(x) if sign < 0 else n * np.fft.ifft(x)
    for a in range(0, t + 1):
        r, c = 1 << a, 1 << (t - a)
        assert rel_l2(oracle.fft_four_step(x, r, c, sign), ref) < 1e-13, (r, c)


def test_four_step_full_size_split(oracle):
    # the 2^24 = 4096 x 4096 lift itself, against the radix-2 loop
    n = 1 << 24
    x = rand_c(n, 24)
    assert rel_l2(oracle.fft_four_step(x, 4096, 4096, -1), oracle.fft_radix2(x, -1)) < 1e-13


# -- Appendix B: Omega along each axis --------------------------------------

@pytest.mark.parametrize("shape", [(2, 2), (8, 16), (64, 32), (4, 8, 16), (16, 16, 16), (2, 4, 2, 8)])
def test_nd_matches_numpy_and_onehot(oracle, shape):
    d = len(shape)
    rng = np.random.default_rng(800 + sum(shape))
    x = rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)
    assert rel_l2(oracle.fft_nd(x, d, -1), np.fft.fftn(x)) < 1e-13
    assert rel_l2(oracle.fft_nd(x, d, +1), np.prod(shape) * np.fft.ifftn(x)) < 1e-13
    # separability: an outer product of 1-D exponentials is a one-hot bin
    f = [(3 * s) // 4 for s in shape]
    e = np.ones(shape, complex)
    for ax, (s, fa) in enumerate(zip(shape, f)):
        v = np.exp(2j * np.pi * ((fa * np.arange(s)) % s) / s)
        e = e * v.reshape([s if i == ax else 1 for i in range(d)])
    y = oracle.fft_nd(e, d, -1)
    expect = np.zeros(shape, complex)
    expect[tuple(f)] = np.prod(shape)
    assert np.max(np.abs(y - expect)) < 1e-10


def test_nd_batch_is_independent(oracle):
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, (3, 8, 4)) + 1j * rng.uniform(-1, 1, (3, 8, 4))
    y = oracle.fft_nd(x, 2, -1)
    for b in range(3):
        assert rel_l2(y[b], oracle.fft_nd(x[b], 2, -1)) < 1e-15


# -- Appendix A.1: psi / gamma worked example ---------------------------------

def _read_golden():
    shape, cases = None, []
    with open(os.path.join(GOLDEN, "psi_example.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, _, rest = line.partition(" ")
            if head == "shape":
                shape = [int(v) for v in rest.split()]
            else:
                idx, _, vals = rest.partition("=")
                cases.append((head, [int(v) for v in idx.split()], [int(v) for v in vals.split()]))
    return shape, cases


def test_psi_worked_example(oracle):
    shape, cases = _read_golden()
    A = np.arange(int(np.prod(shape))).reshape(shape)
    for kind, idx, vals in cases:
        if kind == "psi":
            got = np.asarray(oracle.psi(A, idx)).reshape(-1)
        else:
            # Eq. A.3: <1 2> psi (2 take reverse A); reverse acts on axis 0
            # (Definition A.5) and take keeps the first 2 items (Definition A.4)
            taken = A[::-1][:2]
            got = np.asarray(oracle.psi(taken, idx)).reshape(-1)
            assert list(got) == list(np.asarray(oracle.psi(A, idx)).reshape(-1))
        assert list(got) == vals, (kind, idx)
    # the gamma recurrence on the full index <2 1 3>
    assert oracle.gamma(shape, [2, 1, 3]) == 47


# -- the gradient of the differentiation workload (closed form) -------------

def test_gradient_closed_form_matches_central_differences(oracle):
    """L(x) = sum |H * F x|^2 has the gradient dL/dRe + i dL/dIm =
    2 F^H (|H|^2 * F x), F^H being the sign +1 transform.  L is quadratic, so
    FP64 central differences are exact up to rounding: at n = 2^8 they pin the
    closed form that the GPU gradient tests use."""
    from paper_0811_2535_gb300 import inputs
    n = 1 << 8
    H, x = inputs.spectral_filter(n, 1, inputs.SEED_GRADIENT)
    H = H.astype(np.complex128)
    x = x.reshape(n).astype(np.complex128)

    def loss(v):
        return float(np.sum(np.abs(H * oracle.fft_radix2(v, -1)) ** 2))

    h = 1e-3
    fd = np.empty(n, np.complex128)
    for j in range(n):
        parts = []
        for unit in (1.0, 1j):
            xp, xm = x.copy(), x.copy()
            xp[j] += h * unit
            xm[j] -= h * unit
            parts.append((loss(xp) - loss(xm)) / (2 * h))
        fd[j] = parts[0] + 1j * parts[1]
    closed = 2.0 * oracle.fft_radix2(np.abs(H) ** 2 * oracle.fft_radix2(x, -1), +1)
    assert rel_l2(closed, fd) < 1e-9
    # a dropped factor 2 or the forward transform in place of F^H fails
    assert rel_l2(oracle.fft_radix2(np.abs(H) ** 2 * oracle.fft_radix2(x, -1), +1), fd) > 0.4
    assert rel_l2(2.0 * oracle.fft_radix2(np.abs(H) ** 2 * oracle.fft_radix2(x, -1), -1), fd) > 0.4
