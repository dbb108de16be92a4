"""FP64 CPU oracle for the MoA reshape-transpose FFT (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is a thin ctypes wrapper over
``fft_oracle.c`` (plain C, FP64) and shares nothing with the CUDA path.

Conventions (the same in every function): complex128 numpy arrays,
row-major, batch outermost, unnormalised, exponent sign ``sign`` in
{-1, +1}: ``X[k] = sum_j x[j] exp(sign * 2 pi i j k / n)``.

Which passage each function follows:

* :func:`dft_naive`      -- the DFT definition (Fig. 2.1, "Output").
* :func:`fft_radix2`     -- Fig. 2.1 bit reversal + Sec. 3.5-3.6 in-place
  radix-2 butterfly loop, weights per stage as in Fig. 3.8.
* :func:`fft_partitioned` -- Sec. 4.2-4.8, Fig. 4.9 block/cyclic plan split
  at ``breakpoint`` over ``m`` processors.
* :func:`fft_four_step`  -- dimension lifting n = r*c (column DFTs, twiddle,
  row DFTs, transposed output).
* :func:`fft_nd`         -- Appendix B, Eq. B.6 (Omega along each axis).
* :func:`gamma`          -- Appendix A, Definition A.1 (row-major offset).

The paper's shared-memory all-processor templates, run on the host cores
(``fft_template.c``, OpenMP where gcc has it), are the CPU comparison point
for the GPU path; their results equal the sequential plans bit for bit:

* :func:`template_partitioned` -- Sec. 6.3, Fig. 6.4 (both p loops parallel).
* :func:`template_nd`          -- Eq. B.6 with the lines of each axis in
  parallel.

Every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` against brute force, closed forms, invariants
and the worked example of Appendix A.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fft_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
_TSRC = os.path.join(_HERE, "fft_template.c")
_TLIB = os.path.join(_HERE, "libtemplate.so")
_tlib = None


def build(force: bool = False) -> str:
    """Compile ``fft_oracle.c`` into ``liboracle.so`` with gcc (no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fno-fast-math", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def build_template(force: bool = False) -> str:
    """Compile ``fft_template.c`` into ``libtemplate.so``: with OpenMP where the
    compiler accepts ``-fopenmp``, else as plain sequential C."""
    if force or not os.path.exists(_TLIB) or os.path.getmtime(_TLIB) < os.path.getmtime(_TSRC):
        tmp = _TLIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fno-fast-math", "-shared", "-fPIC", "-o", tmp, _TSRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except (subprocess.CalledProcessError, OSError):
            subprocess.check_call(base)
        os.replace(tmp, _TLIB)
    return _TLIB


def _load_template():
    global _tlib
    if _tlib is None:
        lib = ctypes.CDLL(build_template())
        dp = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        lib.tmpl_fft_partitioned.argtypes = [dp, i64, i64, ctypes.c_int, ctypes.c_int]
        lib.tmpl_fft_nd.argtypes = [dp, ctypes.POINTER(i64), ctypes.c_int, i64, ctypes.c_int]
        lib.tmpl_max_threads.argtypes = []
        for f in ("tmpl_fft_partitioned", "tmpl_fft_nd", "tmpl_max_threads"):
            getattr(lib, f).restype = ctypes.c_int
        _tlib = lib
    return _tlib


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        lib.oracle_dft_naive.argtypes = [dp, dp, i64, ctypes.c_int]
        lib.oracle_fft_radix2.argtypes = [dp, i64, ctypes.c_int]
        lib.oracle_fft_radix2_batch.argtypes = [dp, i64, i64, ctypes.c_int]
        lib.oracle_fft_partitioned.argtypes = [dp, i64, i64, ctypes.c_int, ctypes.c_int]
        lib.oracle_fft_four_step.argtypes = [dp, dp, i64, i64, ctypes.c_int]
        lib.oracle_fft_nd.argtypes = [dp, ctypes.POINTER(i64), ctypes.c_int, i64, ctypes.c_int]
        lib.oracle_gamma.argtypes = [ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.c_int]
        lib.oracle_gamma.restype = i64
        for f in ("oracle_dft_naive", "oracle_fft_radix2", "oracle_fft_radix2_batch",
                  "oracle_fft_partitioned", "oracle_fft_four_step", "oracle_fft_nd"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what}: invalid argument (code {rc})")


def dft_naive(x, sign: int = -1) -> np.ndarray:
    """O(n^2) DFT of a 1-D vector, exponent reduced exactly mod n."""
    x = _c128(x)
    y = np.empty_like(x)
    _check(_load().oracle_dft_naive(_ptr(x), _ptr(y), x.size, sign), "dft_naive")
    return y


def fft_radix2(x, sign: int = -1) -> np.ndarray:
    """Fig. 2.1 / Sec. 3.6 radix-2 FFT along the last axis (any leading batch)."""
    y = _c128(x).copy()
    n = y.shape[-1]
    _check(_load().oracle_fft_radix2_batch(_ptr(y), n, y.size // n if n else 0, sign), "fft_radix2")
    return y


def fft_partitioned(x, m: int, breakpoint: int, sign: int = -1) -> np.ndarray:
    """Fig. 4.9 combined block/cyclic plan (1-D vector)."""
    y = _c128(x).copy()
    _check(_load().oracle_fft_partitioned(_ptr(y), y.size, m, breakpoint, sign), "fft_partitioned")
    return y


def fft_four_step(x, r: int, c: int, sign: int = -1) -> np.ndarray:
    """Dimension-lifting form n = r*c (1-D vector)."""
    x = _c128(x)
    if x.size != r * c:
        raise ValueError("r*c must equal the vector length")
    y = np.empty_like(x)
    _check(_load().oracle_fft_four_step(_ptr(x), _ptr(y), r, c, sign), "fft_four_step")
    return y


def fft_nd(x, dims: int, sign: int = -1) -> np.ndarray:
    """DFT over the last ``dims`` axes (Omega along each), leading axes = batch."""
    y = _c128(x).copy()
    shape = y.shape[y.ndim - dims:]
    batch = int(np.prod(y.shape[:y.ndim - dims], dtype=np.int64)) if y.ndim > dims else 1
    sh = (ctypes.c_int64 * dims)(*shape)
    _check(_load().oracle_fft_nd(_ptr(y), sh, dims, batch, sign), "fft_nd")
    return y


def gamma(shape, index) -> int:
    """Row-major offset of a full index (Definition A.1)."""
    d = len(shape)
    sh = (ctypes.c_int64 * d)(*shape)
    ix = (ctypes.c_int64 * d)(*index)
    return int(_load().oracle_gamma(sh, ix, d))


def psi(a: np.ndarray, index) -> np.ndarray:
    """``index psi A`` for a full or partial index (Definition A.1), via gamma
    on the vector of items of ``a`` (row-major)."""
    shape = list(a.shape)
    k = len(index)
    flat = np.asarray(a).reshape(-1)
    rest = shape[k:]
    count = int(np.prod(rest, dtype=np.int64)) if rest else 1
    start = gamma(shape, list(index) + [0] * (len(shape) - k))
    out = flat[start:start + count]
    return out.reshape(rest) if rest else out[0]


def template_threads() -> int:
    """Threads the parallel loops of the templates use (1 without OpenMP)."""
    return int(_load_template().tmpl_max_threads())


def template_partitioned(x, m: int, breakpoint: int, sign: int = -1) -> np.ndarray:
    """Fig. 6.4: the Fig. 4.9 plan with both p loops run in parallel (1-D)."""
    y = _c128(x).copy()
    _check(_load_template().tmpl_fft_partitioned(_ptr(y), y.size, m, breakpoint, sign),
           "template_partitioned")
    return y


def template_nd(x, dims: int, sign: int = -1, inplace: bool = False) -> np.ndarray:
    """Eq. B.6 over the last ``dims`` axes with the lines of each axis run in
    parallel; leading axes are the batch.  ``inplace`` transforms a contiguous
    complex128 ``x`` itself."""
    y = x if inplace else _c128(x).copy()
    if inplace and not (y.dtype == np.complex128 and y.flags.c_contiguous):
        raise ValueError("inplace needs a contiguous complex128 array")
    shape = y.shape[y.ndim - dims:]
    batch = int(np.prod(y.shape[:y.ndim - dims], dtype=np.int64)) if y.ndim > dims else 1
    sh = (ctypes.c_int64 * dims)(*shape)
    _check(_load_template().tmpl_fft_nd(_ptr(y), sh, dims, batch, sign), "template_nd")
    return y
