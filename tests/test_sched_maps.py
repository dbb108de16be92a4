"""Index maps of the in-register stages (CPU).

The GPU kernels move data by index formulas that their source states in
comments; this file restates those formulas in plain numpy and checks, for
every length and radix schedule, that they compute the DFT (numpy's FFT as
the reference).  A failing GPU parity test can then be traced either to the
maps (this file fails too) or to the code that implements them.

  Stockham stages (fft_core.cuh), schedule V of Sched<L, V>:
    stage s, K = product of earlier radices, M = N/K, M1 = M/R:
    butterfly b = kappa*M1 + u reads e = kappa*M + u + M1*m (m < R),
    y[k] = sum_m x_m w_R^(m k) * w_M^(u k), writes e = (kappa + K*k)*M1 + u;
    thread tau owns butterflies tau + T*i; registers load element
    tau + T*q into (q % NB0)*R0 + q / NB0; after the last stage (radix R)
    register i*R + k holds X[tau + T*(i + (16/R)*k)].
  Warp-shuffle rows (pass_kernels.cu, row_warp_kernel): lane lam of T holds
    element lam + T*q in register q; radix-16 over q, twiddle w_N^(lam k1);
    radix-2 stages across lanes with spans h = T/2 .. 1 (lower lane: sum,
    upper lane: difference times w_2h^(lam mod h)); lane lam then holds
    X[k1 + 16*bitrev(lam)]; staging row = lane, the warp's outputs read back
    at position p = lane + 32*m."""
import numpy as np
import pytest


def radix_logs(L, V):
    if V == 2:
        S = 1 if L <= 3 else (L + 2) // 3
        return [L] if L <= 3 else [(L % 3) if (s == 0 and L % 3) else 3 for s in range(S)]
    if L <= 4:
        return [L]
    S = (L + 3) // 4
    if V == 1:
        return [(L % 4) if (s == S - 1 and L % 4) else 4 for s in range(S)]
    return [(L % 4) if (s == 0 and L % 4) else 4 for s in range(S)]


def exists(L, V):
    if V == 0:
        return 1 <= L <= 12
    if V == 1:
        return 9 <= L <= 11
    return 7 <= L <= 12


def schedule_valid(L, V):
    """Every stage but the last writes at offsets (N/R)*k that are multiples
    of 16 (the padded exchange's base-plus-offset addressing)."""
    N, rl = 1 << L, radix_logs(L, V)
    return all(((N >> r) % 16) == 0 for r in rl[:-1])


def pad16(e):
    return e + (e >> 4)


def stockham(x, V):
    N = x.size
    L = N.bit_length() - 1
    P = min(N, 16)
    T = N // P
    rl = radix_logs(L, V)
    R0 = 1 << rl[0]
    NB0 = P // R0
    v = np.zeros((T, P), complex)
    for tau in range(T):
        for q in range(P):
            v[tau, (q % NB0) * R0 + q // NB0] = x[tau + T * q]
    K = 1
    prev = None
    for s, r in enumerate(rl):
        R = 1 << r
        NB = P // R
        M1 = N // K // R
        M = M1 * R
        if s > 0:
            Rp = 1 << prev
            sm = {}
            for tau in range(T):
                for i in range(P // Rp):
                    b = tau + T * i
                    for k in range(Rp):
                        e = b + (N // Rp) * k
                        # the padded slot of base plus offset equals the slot of the element
                        assert pad16(b) + pad16((N // Rp) * k) == pad16(e)
                        sm[e] = v[tau, i * Rp + k]
            for tau in range(T):
                for i in range(NB):
                    b = tau + T * i
                    w = (b // M1) * M + (b % M1)
                    for m in range(R):
                        assert pad16(w) + pad16(M1 * m) == pad16(w + M1 * m)
                        v[tau, i * R + m] = sm[w + M1 * m]
        for tau in range(T):
            for i in range(NB):
                b = tau + T * i
                u = b % M1
                blk = v[tau, i * R:(i + 1) * R]
                y = np.fft.fft(blk)
                if s != len(rl) - 1:
                    y = y * np.exp(-2j * np.pi * u * np.arange(R) / M)
                v[tau, i * R:(i + 1) * R] = y
        K *= R
        prev = r
    RL = 1 << rl[-1]
    NBL = P // RL
    out = np.zeros(N, complex)
    for tau in range(T):
        for i in range(NBL):
            for k in range(RL):
                out[tau + T * (i + NBL * k)] = v[tau, i * RL + k]
    return out


@pytest.mark.parametrize("V", [0, 1, 2])
@pytest.mark.parametrize("L", range(1, 13))
def test_stockham_maps_compute_the_dft(L, V):
    if not exists(L, V):
        pytest.skip("schedule not defined for this length")
    assert schedule_valid(L, V)
    assert sum(radix_logs(L, V)) == L
    x = np.random.default_rng(L * 10 + V).standard_normal((1 << L, 2)) @ np.array([1, 1j])
    err = np.abs(stockham(x, V) - np.fft.fft(x)).max() / np.abs(np.fft.fft(x)).max()
    assert err < 1e-12


def test_schedules_exist_exactly_where_valid():
    """The lengths on which the plan offers schedules 1 and 2 are lengths on
    which they are valid and differ from schedule 0."""
    for L in range(1, 13):
        for V in (1, 2):
            if exists(L, V):
                assert schedule_valid(L, V) and radix_logs(L, V) != radix_logs(L, 0), (L, V)


def bitrev(x, bits):
    r = 0
    for _ in range(bits):
        r = (r << 1) | (x & 1)
        x >>= 1
    return r


def warp_rows(X):
    """The warp-shuffle kernel on rows X (O x N), warp by warp."""
    O, N = X.shape
    T = N // 16
    LT = T.bit_length() - 1
    per_warp = 32 // T
    out = np.full_like(X, np.nan)
    for o0 in range(0, O, per_warp):
        v = np.zeros((32, 16), complex)
        for lane in range(32):
            g, lam = divmod(lane, T)
            if o0 + g < O:
                v[lane] = X[o0 + g, lam + T * np.arange(16)]
        for lane in range(32):
            lam = lane % T
            v[lane] = np.fft.fft(v[lane]) * np.exp(-2j * np.pi * lam * np.arange(16) / N)
        h = T // 2
        while h >= 1:
            nv = v.copy()
            for lane in range(32):
                lam = lane % T
                p = v[lane ^ h]
                if lam & h:
                    nv[lane] = (p - v[lane]) * np.exp(-2j * np.pi * (lam % h) * (T // (2 * h)) / T)
                else:
                    nv[lane] = v[lane] + p
            v = nv
            h //= 2
        for m in range(16):
            for lane in range(32):
                p = lane + 32 * m
                fl, k = p // N, p % N
                if o0 + fl < O:
                    out[o0 + fl, k] = v[fl * T + bitrev(k >> 4, LT), k & 15]
    return out


@pytest.mark.parametrize("L", [7, 8, 9])
@pytest.mark.parametrize("O", [1, 5])
def test_warp_shuffle_maps_compute_the_dft(L, O):
    X = np.random.default_rng(L + O).standard_normal((O, 1 << L, 2)) @ np.array([1, 1j])
    ref = np.fft.fft(X, axis=1)
    assert np.abs(warp_rows(X) - ref).max() / np.abs(ref).max() < 1e-12


def test_warp_staging_reads_are_conflict_free():
    """The staged outputs are read back with 17 complex64 per row: within a
    half-warp (8-byte accesses) the sixteen lanes hit sixteen different bank
    pairs, for every T and read step m."""
    for L in (7, 8, 9):
        N, T = 1 << L, 1 << (L - 4)
        LT = L - 4
        for m in range(16):
            for half in (0, 1):
                banks = []
                for lane in range(16 * half, 16 * half + 16):
                    p = lane + 32 * m
                    fl, k = p // N, p % N
                    slot = (fl * T + bitrev(k >> 4, LT)) * 17 + (k & 15)
                    banks.append((2 * slot) % 32)
                assert len(set(banks)) == 16, (L, m, half)
