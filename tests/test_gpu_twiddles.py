"""Twiddle tables (GPU): every FP32 entry of a plan's tables is the FP64
value w_M^e = exp(-2 pi i e / M) rounded once, to within 1 ulp per component
(the two FP64 evaluations, the device's and this file's, may fall on either
side of an FP32 rounding boundary), and the four-step twiddle formed in the
kernels as the product of the two halves stays within a few FP32 ulps.

The reference here is independent of the device code: the exponent is
reduced exactly to a quadrant (so multiples of a quarter turn give exact 0
and +-1) and the remaining angle, below pi/2, goes to numpy's FP64 cos/sin.
The stage layout is restated from the documented schedule: a stage of radix
2^(L mod 4) first when L is not a multiple of 4, radix 16 after that; the
table holds rows k = 1, 2, 3, 4, 8, 12 of w_M^(u k), u < M1, for every stage
but the last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def moafft():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0811_2535_gb300 import build, moafft as m
    build.build()
    return m


def root64(e, M):
    """exp(-2 pi i e / M) in FP64 for integer arrays e, power-of-two M."""
    e = np.asarray(e, dtype=np.int64) % M
    q, r = np.divmod(4 * e, M)                 # quadrant, remainder (units of 1/(4M) turn)
    theta = (np.pi / 2) * (r.astype(np.float64) / M)
    c0, s0 = np.cos(theta), np.sin(theta)
    c0 = np.where(r == 0, 1.0, c0)
    s0 = np.where(r == 0, 0.0, s0)
    c = np.select([q == 0, q == 1, q == 2, q == 3], [c0, -s0, -c0, s0])
    s = np.select([q == 0, q == 1, q == 2, q == 3], [s0, c0, -s0, -c0])
    return c - 1j * s


def ordered(x):
    """FP32 values mapped to integers in the order of the reals (+0 = -0)."""
    i = np.ascontiguousarray(x, dtype=np.float32).view(np.int32).astype(np.int64)
    return np.where(i < 0, -(i & 0x7FFFFFFF), i)


def ulps(a32, ref64):
    a = np.asarray(a32, dtype=np.complex64)
    r = ref64.astype(np.complex64)
    return np.maximum(np.abs(ordered(a.real) - ordered(r.real)), np.abs(ordered(a.imag) - ordered(r.imag)))


def stage_reference(L):
    N = 1 << L
    if L <= 4:
        return np.zeros(0, np.complex128)
    S = (L + 3) // 4
    radix_log = [(L % 4) if (s == 0 and L % 4) else 4 for s in range(S)]
    parts, K = [], 1
    for s in range(S - 1):
        R = 1 << radix_log[s]
        M1 = N // K // R
        M = M1 * R
        u = np.arange(M1, dtype=np.int64)
        for k in (1, 2, 3, 4, 8, 12):
            parts.append(root64(u * k, M))
        K *= R
    return np.concatenate(parts)


def test_reference_special_values():
    w = root64(np.array([0, 1, 2, 3]), 4)
    assert np.array_equal(w, np.array([1, -1j, -1, 1j]))
    assert np.max(np.abs(root64(np.arange(64), 64) - np.exp(-2j * np.pi * np.arange(64) / 64))) < 1e-15


@pytest.mark.parametrize("L", range(5, 13))
def test_stage_tables_correctly_rounded(moafft, L):
    plan = moafft.Plan([1 << L], 1, -1)
    t = plan.table(0, L)
    plan.destroy()
    ref = stage_reference(L)
    assert t.shape == ref.shape
    assert ulps(t, ref).max() <= 1


@pytest.mark.parametrize("L", [13, 16, 20, 24])
def test_four_step_halves_and_product(moafft, L, monkeypatch):
    monkeypatch.setenv("MOA_AUTOTUNE", "0")
    n = 1 << L
    plan = moafft.Plan([n], 1, -1)
    lo, hi = plan.table(1), plan.table(2)
    stage = plan.table(0, plan.info()["split_r"].bit_length() - 1)
    plan.destroy()
    h = lo.size.bit_length() - 1
    assert lo.size * hi.size == n
    assert ulps(lo, root64(np.arange(lo.size), n)).max() <= 1
    assert ulps(hi, root64(np.arange(hi.size) << h, n)).max() <= 1
    assert stage.size > 0
    # the kernels' twiddle w_n^e = lo[e mod 2^h] * hi[e >> h], in FP32
    rng = np.random.default_rng(L)
    e = rng.integers(0, n, size=1 << 18)
    w = lo[e & (lo.size - 1)] * hi[e >> h]
    err = np.abs(w.astype(np.complex128) - root64(e, n))
    assert err.max() <= 4 * 2.0 ** -24, err.max()


def test_tables_absent_or_invalid(moafft):
    plan = moafft.Plan([1 << 10], 1, -1)   # one tile: no four-step halves, no stage table of 2^11
    with pytest.raises(moafft.MoaError):
        plan.table(1)
    with pytest.raises(moafft.MoaError):
        plan.table(0, 11)
    with pytest.raises(moafft.MoaError):
        plan.table(3)
    plan.destroy()
