"""Seeded synthetic inputs for the FFT workloads (shared by tests and bench).

This module holds no transform arithmetic: it only draws numbers.  Every
generator uses ``numpy.random.default_rng(seed)``, draws in FP64 and rounds
once to complex64 (the plain FP32 path's storage type); the oracle is then
fed the complex64 values promoted back to FP64, so a parity error measures
the transform alone.  For every complex block the real parts are drawn
first, then the imaginary parts.

Workloads (sizes as in the paper's experiments, Sec. 7.2, n = 2^3..2^24,
extended to the multi-D, batched, precision and gradient cases):

* ``uniform(shape, seed)``          re, im ~ U[-1, 1)
* ``uneven_batch(count, seed)``     lengths 2^k, k ~ U{6..16}, then each
                                    transform's re, im ~ N(0, 1) in order
* ``sinusoids(batch, n, seed)``     U[-1, 1) plus 5 complex sinusoids of
                                    amplitude 10 per transform, distinct
                                    integer frequencies, phases ~ U[0, 1)
* ``spectral_filter(n, batch, seed)`` H ~ N(0,1) (shape [n]) drawn first,
                                    then x ~ U[-1, 1) of shape [batch, n]
"""
from __future__ import annotations

import numpy as np

SEED_SMALL = 0        # 1-D n = 2^10
SEED_LARGE = 1        # 1-D n = 2^24, 2-D 4096^2, 3-D 256^3
SEED_UNEVEN = 2       # 4096 transforms of uneven lengths
SEED_PRECISION = 3    # 16384 x 4096 with sinusoids
SEED_GRADIENT = 4     # spectral filter H and x


def _complex(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    out = np.empty(re.shape, dtype=np.complex64)
    out.real = re.astype(np.float32)
    out.imag = im.astype(np.float32)
    return out


def uniform(shape, seed: int) -> np.ndarray:
    """complex64 array, re and im iid U[-1, 1)."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in (shape if hasattr(shape, "__len__") else (shape,)))
    re = rng.uniform(-1.0, 1.0, size=shape)
    im = rng.uniform(-1.0, 1.0, size=shape)
    return _complex(re, im)


def uneven_lengths(count: int, seed: int = SEED_UNEVEN, kmin: int = 6, kmax: int = 16) -> np.ndarray:
    """The exponents k of the uneven batch (first draw of the generator)."""
    rng = np.random.default_rng(seed)
    return rng.integers(kmin, kmax + 1, count)


def uneven_batch(count: int, seed: int = SEED_UNEVEN, kmin: int = 6, kmax: int = 16):
    """Lengths 2^k (k ~ U{kmin..kmax}) and one complex64 vector per length,
    re then im ~ N(0, 1), drawn transform by transform from the same
    generator.  Returns (lengths int64 array, list of arrays)."""
    rng = np.random.default_rng(seed)
    ks = rng.integers(kmin, kmax + 1, count)
    lengths = (np.int64(1) << ks.astype(np.int64))
    vecs = []
    for n in lengths:
        re = rng.standard_normal(int(n))
        im = rng.standard_normal(int(n))
        vecs.append(_complex(re, im))
    return lengths, vecs


def sinusoids(batch: int, n: int, seed: int = SEED_PRECISION, count: int = 5, amplitude: float = 10.0):
    """[batch, n] complex64: U[-1,1) noise plus ``count`` complex sinusoids
    amplitude*exp(2 pi i (f j / n + phi)) per transform, with distinct
    integer f ~ U{0..n-1} and phi ~ U[0, 1).  Draw order: all noise (re then
    im), then per transform the frequencies and phases."""
    rng = np.random.default_rng(seed)
    re = rng.uniform(-1.0, 1.0, size=(batch, n))
    im = rng.uniform(-1.0, 1.0, size=(batch, n))
    for b in range(batch):
        f = rng.choice(n, size=count, replace=False)
        phi = rng.uniform(0.0, 1.0, size=count)
        # integer phase f*j reduced mod n before scaling keeps the angle exact
        ang = 2.0 * np.pi * (((f[:, None].astype(np.int64) * np.arange(n, dtype=np.int64)[None, :]) % n) / n
                             + phi[:, None])
        re[b] += amplitude * np.cos(ang).sum(axis=0)
        im[b] += amplitude * np.sin(ang).sum(axis=0)
    return _complex(re, im)


def spectral_filter(n: int, batch: int, seed: int = SEED_GRADIENT):
    """(H [n] complex64 ~ N(0,1), x [batch, n] complex64 ~ U[-1,1)), H first."""
    rng = np.random.default_rng(seed)
    hre = rng.standard_normal(n)
    him = rng.standard_normal(n)
    xre = rng.uniform(-1.0, 1.0, size=(batch, n))
    xim = rng.uniform(-1.0, 1.0, size=(batch, n))
    return _complex(hre, him), _complex(xre, xim)
