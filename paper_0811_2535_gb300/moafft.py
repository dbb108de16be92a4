"""Python binding of libmoafft.so (the C ABI in include/moa_fft.h).

Argument marshalling only: every transform runs in the library's CUDA
kernels.  PyTorch supplies device memory (``tensor.data_ptr()``) and the
stream (``torch.cuda.current_stream().cuda_stream``).  There is no CPU or
library fallback: if the shared library is missing or cannot be loaded the
first call raises.

Conventions follow the C ABI: complex64, row-major, batch outermost,
unnormalised, ``sign`` in {-1, +1} with X[k] = sum_j x[j] exp(sign 2 pi i jk/n).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmoafft.so")

MOA_C64, MOA_C64_TC_FP16, MOA_C64_TC_BF16 = 0, 1, 2
STATUS = {0: "MOA_OK", 1: "MOA_ERR_INVALID_ARG", 2: "MOA_ERR_INVALID_SIZE", 3: "MOA_ERR_UNSUPPORTED",
          4: "MOA_ERR_ALLOC", 5: "MOA_ERR_CUDA", 6: "MOA_ERR_TIMEOUT"}
MOA_OK, MOA_ERR_TIMEOUT = 0, 6

# every symbol the header declares, with (restype, argtypes)
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
SIGNATURES = {
    "moa_fft_plan": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(_I64), ctypes.c_int, _I64,
                                    ctypes.c_int, ctypes.c_int]),
    "moa_fft_plan_batched": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(_I64), _I64, ctypes.c_int,
                                            ctypes.c_int]),
    "moa_fft_exec": (ctypes.c_int, [_P, _P, _P, _P]),
    "moa_fft_exec_adjoint": (ctypes.c_int, [_P, _P, _P, _P]),
    "moa_fft_exec_pass": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P]),
    "moa_fft_exec_host": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "moa_fft_exec_noalloc": (ctypes.c_int, [_P, _P, _I64, ctypes.c_int, _P]),
    "moa_fft_noalloc_status": (ctypes.c_int, [_P]),
    "moa_fft_status": (ctypes.c_int, [_P]),
    "moa_fft_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "moa_fft_plan_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_I64),
                                         ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_size_t)]),
    "moa_fft_pass_info": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(_I64)]),
    "moa_fft_plan_choice": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_size_t]),
    "moa_fft_estimate": (ctypes.c_int, [ctypes.POINTER(_I64), ctypes.c_int, _I64, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                        ctypes.POINTER(ctypes.c_size_t), ctypes.c_char_p, ctypes.c_size_t]),
    "moa_fft_plan_table": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _I64, ctypes.POINTER(_I64)]),
    "moa_fft_batched_queue": (ctypes.c_int, [ctypes.POINTER(_I64), _I64, _I64, ctypes.POINTER(_I64),
                                             ctypes.POINTER(ctypes.c_int32), _I64, ctypes.POINTER(_I64)]),
    "moa_fft_destroy": (ctypes.c_int, [_P]),
}

_lib = None


class MoaError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)} ({error_string(code) if _lib else ''})")


def lib() -> ctypes.CDLL:
    """Load libmoafft.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmoafft.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def estimate(shape: Sequence[int], batch: int = 1, dtype: int = MOA_C64, tma: int = -1) -> dict:
    """Host-only description of the plan for ``shape`` x ``batch`` with the
    autotuner off (``moa_fft_estimate``): passes, r x c split, workspace bytes
    and the kernel of each pass.  ``tma``: 1 / 0 assume the tensor-map encoder
    present / absent, -1 asks the driver.  Needs no GPU."""
    arr = (_I64 * len(shape))(*[int(v) for v in shape])
    np_, r, c, ws = ctypes.c_int(), _I64(), _I64(), ctypes.c_size_t()
    buf = ctypes.create_string_buffer(512)
    _check(lib().moa_fft_estimate(arr, len(shape), int(batch), int(dtype), int(tma), ctypes.byref(np_),
                                  ctypes.byref(r), ctypes.byref(c), ctypes.byref(ws), buf, len(buf)),
           "moa_fft_estimate")
    return {"passes": np_.value, "split_r": r.value, "split_c": c.value, "workspace_bytes": ws.value,
            "kernels": buf.value.decode().split(";") if buf.value else []}


def batched_queue(lengths: Sequence[int], resident: int):
    """Host-only work queue of a batched plan (``moa_fft_batched_queue``):
    returns (order, tasks) with tasks an (ntasks, 6) int32 array of rows
    {first, count, tile, log2 n, log2 r, kind}.  Needs no GPU."""
    import numpy as np
    arr = (_I64 * len(lengths))(*[int(v) for v in lengths])
    nt = _I64()
    _check(lib().moa_fft_batched_queue(arr, len(lengths), int(resident), None, None, 0, ctypes.byref(nt)),
           "moa_fft_batched_queue")
    order = np.empty(len(lengths), dtype=np.int64)
    tasks = np.empty((nt.value, 6), dtype=np.int32)
    _check(lib().moa_fft_batched_queue(arr, len(lengths), int(resident),
                                       order.ctypes.data_as(ctypes.POINTER(_I64)),
                                       tasks.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), nt.value,
                                       ctypes.byref(nt)), "moa_fft_batched_queue")
    return order, tasks


def error_string(code: int) -> str:
    return lib().moa_fft_error_string(code).decode()


def _check(code: int, what: str) -> None:
    if code != 0:
        raise MoaError(code, what)


def _stream_ptr(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Plan:
    """A plan for ``batch`` transforms of ``shape`` (1-, 2- or 3-D)."""

    def __init__(self, shape: Sequence[int], batch: int = 1, sign: int = -1, dtype: int = MOA_C64):
        shape = [int(s) for s in (shape if hasattr(shape, "__len__") else [shape])]
        self.shape, self.batch, self.sign, self.dtype = tuple(shape), int(batch), int(sign), int(dtype)
        arr = (_I64 * len(shape))(*shape)
        h = _P()
        _check(lib().moa_fft_plan(ctypes.byref(h), arr, len(shape), self.batch, self.sign, self.dtype),
               f"moa_fft_plan{tuple(shape)}x{batch}")
        self._h = h

    @property
    def numel(self) -> int:
        n = self.batch
        for s in self.shape:
            n *= s
        return n

    def _io(self, x, out):
        import torch
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.complex64):
            raise TypeError("input must be a complex64 CUDA tensor")
        if not x.is_contiguous():
            x = x.contiguous()
        if x.numel() != self.numel:
            raise ValueError(f"input has {x.numel()} elements, plan expects {self.numel}")
        if out is None:
            out = torch.empty_like(x)
        elif not (out.is_cuda and out.dtype == torch.complex64 and out.is_contiguous() and out.numel() == self.numel):
            raise ValueError("out must be a contiguous complex64 CUDA tensor of the plan's size")
        return x, out

    def exec(self, x, out=None, stream=None):
        """Transform ``x`` (complex64 CUDA tensor) into ``out`` (new if None)."""
        x, out = self._io(x, out)
        _check(lib().moa_fft_exec(self._h, x.data_ptr(), out.data_ptr(), _stream_ptr(stream)), "moa_fft_exec")
        return out

    def exec_adjoint(self, x, out=None, stream=None):
        """Opposite-sign unnormalised transform (F^H) on the same plan."""
        x, out = self._io(x, out)
        _check(lib().moa_fft_exec_adjoint(self._h, x.data_ptr(), out.data_ptr(), _stream_ptr(stream)),
               "moa_fft_exec_adjoint")
        return out

    def exec_pass(self, index: int, x, out, sign: Optional[int] = None, stream=None):
        """Run only pass ``index`` (instrumentation: per-kernel timing)."""
        s = self.sign if sign is None else int(sign)
        _check(lib().moa_fft_exec_pass(self._h, int(index), s, x.data_ptr(), out.data_ptr(), _stream_ptr(stream)),
               "moa_fft_exec_pass")
        return out

    def exec_host(self, host_in, host_out, dev_buf, stream=None):
        """Host-memory round trip through ``dev_buf`` (all three torch tensors)."""
        _check(lib().moa_fft_exec_host(self._h, host_in.data_ptr(), host_out.data_ptr(), dev_buf.data_ptr(),
                                       _stream_ptr(stream)), "moa_fft_exec_host")
        return host_out

    def status(self) -> int:
        return lib().moa_fft_status(self._h)

    def info(self) -> dict:
        p = ctypes.c_int()
        r = _I64()
        c = _I64()
        w = ctypes.c_size_t()
        _check(lib().moa_fft_plan_info(self._h, ctypes.byref(p), ctypes.byref(r), ctypes.byref(c), ctypes.byref(w)),
               "moa_fft_plan_info")
        return {"passes": p.value, "split_r": r.value, "split_c": c.value, "workspace_bytes": w.value}

    def choice(self) -> str:
        """The plan's split, tile and kernels, and where they came from."""
        buf = ctypes.create_string_buffer(512)
        _check(lib().moa_fft_plan_choice(self._h, buf, 512), "moa_fft_plan_choice")
        return buf.value.decode()

    def pass_info(self, index: int) -> dict:
        """Kernel name and algorithmic bytes of pass ``index``."""
        buf = ctypes.create_string_buffer(64)
        b = _I64()
        _check(lib().moa_fft_pass_info(self._h, int(index), buf, 64, ctypes.byref(b)), "moa_fft_pass_info")
        return {"kernel": buf.value.decode(), "bytes": b.value}

    def table(self, which: int, index: int = 0):
        """Copy of twiddle table ``which`` (0: stage table of 2^index points,
        1 / 2: low / high half of the four-step twiddle, 3 / 4 / 5: stage
        table of radix schedule 1 / 2 / 3 for 2^index points) as a complex64
        numpy array (``moa_fft_plan_table``)."""
        import numpy as np
        count = _I64()
        _check(lib().moa_fft_plan_table(self._h, int(which), int(index), None, 0, ctypes.byref(count)),
               "moa_fft_plan_table")
        out = np.empty(count.value, dtype=np.complex64)
        _check(lib().moa_fft_plan_table(self._h, int(which), int(index), out.ctypes.data, out.size,
                                        ctypes.byref(count)), "moa_fft_plan_table")
        return out

    def destroy(self) -> None:
        if getattr(self, "_h", None):
            lib().moa_fft_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class BatchedPlan(Plan):
    """Independent 1-D transforms of uneven power-of-two lengths (each in
    [2, 65536]) in one persistent launch.  Transform i occupies the
    contiguous block starting at sum(lengths[:i]) of the input and output."""

    def __init__(self, lengths: Sequence[int], sign: int = -1, dtype: int = MOA_C64):
        lengths = [int(n) for n in lengths]
        self.lengths = tuple(lengths)
        self.shape, self.batch, self.sign, self.dtype = (sum(lengths),), 1, int(sign), int(dtype)
        arr = (_I64 * len(lengths))(*lengths)
        h = _P()
        _check(lib().moa_fft_plan_batched(ctypes.byref(h), arr, len(lengths), self.sign, self.dtype),
               f"moa_fft_plan_batched({len(lengths)} transforms)")
        self._h = h

    def offsets(self):
        out, acc = [], 0
        for n in self.lengths:
            out.append(acc)
            acc += n
        return out


_plan_cache: dict = {}


def _cached_plan(shape, batch, sign):
    key = (tuple(shape), int(batch), int(sign))
    p = _plan_cache.get(key)
    if p is None:
        p = Plan(shape, batch, sign)
        _plan_cache[key] = p
    return p


def fft(x, dims: int = 1, sign: int = -1):
    """Unnormalised DFT of ``x`` (complex64 CUDA tensor) over its last
    ``dims`` axes; leading axes are the batch."""
    shape = tuple(x.shape[x.dim() - dims:])
    batch = 1
    for s in x.shape[:x.dim() - dims]:
        batch *= int(s)
    return _cached_plan(shape, batch, sign).exec(x.contiguous()).view(x.shape)


def _autograd():
    import torch

    class MoaFFTFunction(torch.autograd.Function):
        """y = F x with F the plan's transform; the backward pass applies the
        adjoint kernel.  For a linear map y = F x and a real loss L, PyTorch's
        complex gradient convention gives grad_x = F^H grad_y, and F^H is the
        opposite-sign unnormalised transform on the same plan, so nothing is
        saved for the backward pass."""

        @staticmethod
        def forward(ctx, x, plan):
            ctx.plan = plan
            return plan.exec(x.contiguous()).view(x.shape)

        @staticmethod
        def backward(ctx, g):
            return ctx.plan.exec_adjoint(g.contiguous()).view(g.shape), None

    return MoaFFTFunction


_MoaFFTFunction = None


def MoaFFTFunction():
    global _MoaFFTFunction
    if _MoaFFTFunction is None:
        _MoaFFTFunction = _autograd()
    return _MoaFFTFunction


def fft_autograd(x, plan: Plan):
    """Differentiable transform: ``MoaFFTFunction.apply(x, plan)``."""
    return MoaFFTFunction().apply(x, plan)
