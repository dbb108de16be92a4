"""C ABI checks that need no GPU: the library loads, exports every symbol
include/*.h declares, and rejects bad arguments on the host before any CUDA
call.  The allocation fault is injected on the host (MOA_FAULT_ALLOC)."""
import ctypes
import glob
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_0811_2535_gb300 import build, moafft
    build.build()
    return moafft.lib()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names.update(re.findall(r"MOA_API\s+[\w\s\*]+?\b(moa_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_abi():
    names = declared_symbols()
    for must in ("moa_fft_plan", "moa_fft_exec", "moa_fft_destroy", "moa_fft_exec_adjoint",
                 "moa_fft_plan_batched", "moa_fft_status", "moa_fft_error_string"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    from paper_0811_2535_gb300 import moafft
    for name in declared_symbols():
        assert hasattr(L, name), name
        assert name in moafft.SIGNATURES, f"binding lacks {name}"
    out = subprocess.run(["nm", "-D", "--defined-only", moafft.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in declared_symbols():
        assert name in exported, name


def _plan(L, shape, batch=1, sign=-1, dtype=0):
    arr = (ctypes.c_int64 * len(shape))(*shape)
    h = ctypes.c_void_p(12345)
    rc = L.moa_fft_plan(ctypes.byref(h), arr, len(shape), batch, sign, dtype)
    return rc, h


def test_invalid_sizes_rejected_on_host(L):
    for shape in ([1], [3], [6], [0], [-4], [4, 12], [2, 2, 5]):
        rc, h = _plan(L, shape)
        assert rc == 2, shape           # MOA_ERR_INVALID_SIZE
        assert h.value is None


def test_invalid_args_rejected_on_host(L):
    assert _plan(L, [8], batch=0)[0] == 1
    assert _plan(L, [8], sign=0)[0] == 1
    assert _plan(L, [8], sign=2)[0] == 1
    assert _plan(L, [8], dtype=7)[0] == 1
    arr = (ctypes.c_int64 * 4)(2, 2, 2, 2)
    h = ctypes.c_void_p()
    assert L.moa_fft_plan(ctypes.byref(h), arr, 4, 1, -1, 0) == 1     # dims = 4
    assert L.moa_fft_plan(None, arr, 1, 1, -1, 0) == 1                 # NULL plan pointer
    assert L.moa_fft_plan(ctypes.byref(h), None, 1, 1, -1, 0) == 1     # NULL shape


def test_unsupported_requests(L):
    assert _plan(L, [1 << 31])[0] == 3                 # 1-D beyond 2^30
    assert _plan(L, [1 << 25, 2])[0] == 3              # multi-D axis beyond 2^24
    assert _plan(L, [1 << 24], batch=128)[0] == 3      # more than 2^31 elements
    assert _plan(L, [8], dtype=1)[0] == 3              # tensor-core path: n = 256 or 4096 only
    assert _plan(L, [64, 64], dtype=2)[0] == 3


def test_batched_plan_validation(L):
    h = ctypes.c_void_p()
    lens = (ctypes.c_int64 * 3)(64, 3, 128)
    assert L.moa_fft_plan_batched(ctypes.byref(h), lens, 3, -1, 0) == 2
    assert L.moa_fft_plan_batched(ctypes.byref(h), lens, 0, -1, 0) == 1
    assert L.moa_fft_plan_batched(None, lens, 3, -1, 0) == 1
    big = (ctypes.c_int64 * 2)(64, 1 << 17)
    assert L.moa_fft_plan_batched(ctypes.byref(h), big, 2, -1, 0) == 3      # beyond 2^16: unsupported


def test_dead_handles_and_null(L):
    bogus = ctypes.c_void_p(0xDEAD0)
    assert L.moa_fft_destroy(None) == 0
    assert L.moa_fft_destroy(bogus) == 1
    assert L.moa_fft_exec(bogus, None, None, None) == 1
    assert L.moa_fft_exec_adjoint(bogus, None, None, None) == 1
    assert L.moa_fft_status(bogus) == 1
    assert L.moa_fft_plan_info(bogus, None, None, None, None) == 1
    assert L.moa_fft_plan_table(bogus, 0, 12, None, 0, None) == 1
    assert L.moa_fft_exec_host(bogus, None, None, None, None) == 1
    assert L.moa_fft_exec_pass(bogus, 0, -1, None, None, None) == 1
    assert L.moa_fft_pass_info(bogus, 0, None, 0, None) == 1


def test_error_strings(L):
    for code in range(7):
        s = L.moa_fft_error_string(code)
        assert isinstance(s, bytes) and len(s) > 3
    assert L.moa_fft_error_string(99) == b"unknown status"


def test_allocation_fault_injection():
    # a fresh process so the environment variable is read by the library
    code = (
        "import ctypes, sys; sys.path.insert(0, %r)\n"
        "from paper_0811_2535_gb300 import moafft\n"
        "L = moafft.lib(); h = ctypes.c_void_p(7)\n"
        "arr = (ctypes.c_int64 * 1)(1 << 20)\n"
        "rc = L.moa_fft_plan(ctypes.byref(h), arr, 1, 1, -1, 0)\n"
        "print(rc, h.value)\n" % ROOT
    )
    env = dict(os.environ, MOA_FAULT_ALLOC="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=120)
    assert out.returncode == 0, out.stderr
    rc, hv = out.stdout.split()
    assert int(rc) == 4 and hv == "None"    # MOA_ERR_ALLOC, *plan = NULL


def test_header_enums_match_the_binding(L):
    """The status and dtype values the header declares are the ones the
    binding uses, and every status code has its own description."""
    from paper_0811_2535_gb300 import moafft
    text = open(os.path.join(ROOT, "include", "moa_fft.h")).read()
    declared = {name: int(val) for name, val in re.findall(r"\b(MOA_(?:OK|ERR_\w+|C64\w*))\s*=\s*(\d+)", text)}
    status = {v: k for k, v in declared.items() if k == "MOA_OK" or k.startswith("MOA_ERR_")}
    assert status == moafft.STATUS
    assert (declared["MOA_C64"], declared["MOA_C64_TC_FP16"], declared["MOA_C64_TC_BF16"]) == \
        (moafft.MOA_C64, moafft.MOA_C64_TC_FP16, moafft.MOA_C64_TC_BF16)
    assert (moafft.MOA_OK, moafft.MOA_ERR_TIMEOUT) == (declared["MOA_OK"], declared["MOA_ERR_TIMEOUT"])
    strings = [L.moa_fft_error_string(code).decode() for code in sorted(status)]
    assert len(set(strings)) == len(strings) and all(strings)
    assert L.moa_fft_error_string(99).decode() not in strings[1:]


def test_binding_signatures_match_header_prototypes():
    """Every prototype in include/*.h takes as many arguments as the
    binding's ctypes signature passes, and returns a pointer exactly where
    the binding expects one (the error-string call)."""
    from paper_0811_2535_gb300 import moafft
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for ret, name, params in re.findall(r"MOA_API\s+([\w\s\*]+?)\s*\b(moa_\w+)\s*\(([^)]*)\)", text):
            params = params.strip()
            n = 0 if params in ("", "void") else params.count(",") + 1
            res, args = moafft.SIGNATURES[name]
            assert len(args) == n, (name, n, len(args))
            assert ("*" in ret) == (res is ctypes.c_char_p), (name, ret)
