"""The oracle's pins are not vacuous (CPU only).

Each case plants one plausible mistake in a copy of ``oracle/fft_oracle.c``
(a dropped sign, a wrong root order, a missing stage, a transposed index, a
wrong offset), builds it into a library of its own in a temporary directory
and runs the unchanged pin suite ``tests/test_oracle_pins.py`` against it in a
child process.  Every mutant must make at least one pin fail; the unmodified
copy must pass them all.  The committed oracle is never touched.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_C = os.path.join(ROOT, "oracle", "fft_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (what the mistake is, text, replacement, which occurrence: None = all)
MUTANTS = [
    ("weights lose the exponent sign", "*im = (double)s * sin(a);", "*im = sin(a);", None),
    ("root angle over twice the order", "double a = TWO_PI * ((double)num / (double)den);",
     "double a = TWO_PI * ((double)num / (double)(2 * den));", None),
    ("DFT definition: wrong sign in the imaginary part", "si += xr * wi + xi * wr;", "si += xr * wi - xi * wr;",
     None),
    ("bit reversal P_n left out", "if (j < k) {", "if (j < k && 0) {", None),
    ("butterfly product conjugated (sequential loop)", "double cr = wr * hi[0] - wi * hi[1];",
     "double cr = wr * hi[0] + wi * hi[1];", 0),
    ("butterfly product conjugated (cyclic phase)", "double cr = wr * hi[0] - wi * hi[1];",
     "double cr = wr * hi[0] + wi * hi[1];", 1),
    ("butterfly difference reversed", "hi[0] = dr - cr;", "hi[0] = cr - dr;", 0),
    ("stage weights of order L/2 instead of L", "unit_root(row, L, sign, &weight[2 * row], &weight[2 * row + 1]);",
     "unit_root(row, half, sign, &weight[2 * row], &weight[2 * row + 1]);", None),
    ("cyclic weights without the processor offset p",
     "unit_root(m * rp + p, L, sign, &weight[2 * rp], &weight[2 * rp + 1]);",
     "unit_root(m * rp, L, sign, &weight[2 * rp], &weight[2 * rp + 1]);", None),
    ("cyclic copy without the offset p", "priv[2 * i] = x[2 * (m * i + p)];", "priv[2 * i] = x[2 * (m * i)];", None),
    ("cyclic phase starts one stage late", "for (int q = breakpoint; q <= t; ++q)",
     "for (int q = breakpoint + 1; q <= t; ++q)", None),
    ("block phase stops one stage early", "for (int q = 1; q <= breakpoint - 1; ++q)",
     "for (int q = 1; q < breakpoint - 1; ++q)", None),
    ("four-step twiddle conjugated", "unit_root((j2 * k1) % n, n, sign, &wr, &wi);",
     "unit_root((j2 * k1) % n, n, -sign, &wr, &wi);", None),
    ("four-step columns read as rows", "line[2 * j1] = x[2 * (c * j1 + j2)];",
     "line[2 * j1] = x[2 * (r * j2 + j1)];", None),
    ("four-step output not transposed", "k1 + r * k2", "k2 + c * k1", None),
    ("Omega skips axis 0", "for (int a = dims - 1; a >= 0; --a) {", "for (int a = dims - 1; a >= 1; --a) {", None),
    ("gamma takes the previous extent", "x = x * shape[j] + index[j];", "x = x * shape[j - 1] + index[j];", None),
]


def mutate(src, old, new, which):
    assert old in src, f"mutation site gone: {old!r}"
    if which is None:
        return src.replace(old, new)
    parts = src.split(old)
    assert which < len(parts) - 1
    return old.join(parts[:which + 1]) + new + old.join(parts[which + 1:])


def run_pins(tmp_path, source, monkeypatch):
    """Build `source` (it must compile: a build failure is not a caught
    mistake), then run the pin suite against it; returns the child's exit
    status (0: every pin passed) and the end of its report."""
    import oracle
    src = tmp_path / "fft_oracle.c"
    src.write_text(source)
    monkeypatch.setattr(oracle, "_SRC", str(src))
    monkeypatch.setattr(oracle, "_LIB", str(tmp_path / "liboracle.so"))
    oracle.build(force=True)
    monkeypatch.undo()
    script = (
        "import sys, pytest\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import oracle\n"
        f"oracle._SRC = {str(src)!r}\n"
        f"oracle._LIB = {str(tmp_path / 'liboracle.so')!r}\n"
        f"sys.exit(pytest.main([{PINS!r}, '-x', '-q', '-p', 'no:cacheprovider']))\n")
    res = subprocess.run([sys.executable, "-c", script], cwd=str(tmp_path), capture_output=True, text=True,
                         timeout=600)
    return res.returncode, res.stdout[-2000:]


def test_unmodified_copy_passes_every_pin(tmp_path, monkeypatch):
    rc, out = run_pins(tmp_path, open(ORACLE_C).read(), monkeypatch)
    assert rc == 0, out


@pytest.mark.parametrize("what,old,new,which", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_the_mistake(tmp_path, what, old, new, which, monkeypatch):
    rc, out = run_pins(tmp_path, mutate(open(ORACLE_C).read(), old, new, which), monkeypatch)
    # status 1 and a failed pin in pytest's summary line: a pin caught it
    # (not a crash, not an error in a fixture)
    summary = [ln for ln in out.splitlines() if ln.strip()][-1] if out.strip() else ""
    assert rc == 1 and "1 failed" in summary and "error" not in summary, \
        f"mistake not caught ({what}), pytest status {rc}:\n{out}"
