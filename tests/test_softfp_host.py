"""The integer-path binary64 routines of csrc/softfp64.cuh, compiled for the
host, against the host's IEEE-754 arithmetic.

The GPU test (test_gpu_softfp.py) compares each routine with the hardware
instruction on ~20 million operands.  This CPU test compiles the same header
with the host C++ compiler (the few CUDA intrinsics it uses are supplied by
tests/softfp_host/cuda_runtime.h from their documented semantics) and runs
several hundred million generated operands through it: the full grid of
exponent pairs, the cipher's value range, every adder gap with tie and
sticky bit patterns, cancellations and constructed halfway cases.  The
reference is the definition of the operation, round to nearest with ties to
even (IEEE 754-2019 Sec. 4.3.1), as the host's floating-point unit computes
it.  Mutated copies of the header (a dropped sticky bit, round-half-up,
truncation in place of floor) must fail, so the classes are shown to reach
the rounding logic they are meant to test.  The multiplies by the compile-time
constants 0.01 and RN(8/3) (dmul_const) run beside the general multiply."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HARNESS = os.path.join(ROOT, "tests", "softfp_host", "harness.cpp")
SHIM = os.path.join(ROOT, "tests", "softfp_host")
HEADER = os.path.join(ROOT, "paper_1201_3114_gb300", "csrc", "softfp64.cuh")

SCALE = 8  # about 700 million cases; a few seconds on 8 cores


def _compile(out, header_dir):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    cmd = [cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-pthread", "-I", SHIM, "-I", header_dir,
           HARNESS, "-o", out]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return out


def _run(exe, scale):
    p = subprocess.run([exe, str(scale)], capture_output=True, text=True, timeout=600)
    rows = {}
    for line in p.stdout.splitlines():
        f = line.split()
        rows[(f[0], f[1])] = dict(cases=int(f[2]), fast=int(f[3]), ties=int(f[4]), bad=int(f[5]),
                                  first=" ".join(f[6:]))
    return p.returncode, rows


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("softfp_host")
    return _compile(str(d / "harness"), os.path.dirname(HEADER))


def test_routines_match_ieee_round_to_nearest_even(harness):
    rc, rows = _run(harness, SCALE)
    bad = {k: v for k, v in rows.items() if v["bad"]}
    assert rc == 0 and not bad, bad
    ops = {"add", "sub", "mul", "mul10", "mul28", "floor13", "muldt", "mulbeta", "addkick", "addz"}
    assert {k[0] for k in rows} == ops
    for op in ops:
        cases = sum(v["cases"] for k, v in rows.items() if k[0] == op)
        fast = sum(v["fast"] for k, v in rows.items() if k[0] == op)
        ties = sum(v["ties"] for k, v in rows.items() if k[0] == op)
        assert cases > 10_000_000 and fast > 5_000_000, (op, cases, fast)
        # exact halfway cases handled by the integer path, not the fallback
        assert ties > 100_000, (op, ties)
    # the tie classes run on the integer path
    for op in ("add", "sub"):
        r = rows[(op, "ties")]
        assert r["fast"] > 0.95 * r["cases"] and r["ties"] > 0.25 * r["cases"], r
        # gaps below 32 with tie and sticky patterns reach the integer path
        assert rows[(op, "gap")]["fast"] > 0.4 * rows[(op, "gap")]["cases"]
    r = rows[("floor13", "ties")]
    assert r["fast"] == r["cases"] == r["ties"], r
    # the cipher's own value range stays on the integer path
    for op in ("mul", "mul10", "mul28", "muldt", "mulbeta"):
        assert rows[(op, "cipher")]["fast"] == rows[(op, "cipher")]["cases"]
    # every constructed halfway product of the constant multiplies is one
    for op in ("muldt", "mulbeta"):
        r = rows[(op, "ties")]
        assert r["fast"] == r["cases"] == r["ties"], r
    assert rows[("add", "cipher")]["fast"] > 0.9 * rows[("add", "cipher")]["cases"]
    # the known-order adders: the cipher's kick and z-update operands stay on
    # the integer path, and so do the ordered tie and gap cases
    assert rows[("addkick", "cipher_kick")]["fast"] > 0.99 * rows[("addkick", "cipher_kick")]["cases"]
    assert rows[("addz", "cipher_z")]["fast"] > 0.9 * rows[("addz", "cipher_z")]["cases"]
    for op in ("addkick", "addz"):
        r = rows[(op, "ties")]
        assert r["fast"] > 0.8 * r["cases"] and r["ties"] > 0.2 * r["cases"], (op, r)
        assert rows[(op, "gap")]["fast"] > 0.3 * rows[(op, "gap")]["cases"], op


MUTATIONS = [
    # (what is planted, text replaced, replacement, an (op, class) that must fail)
    ("dmul rounds half up", "const uint32_t up = guard & ((sticky != 0u) | (q0 & 1u));",
     "const uint32_t up = guard;", ("mul", "cipher_consts")),
    ("the constant multiply rounds half up", "const uint32_t up = guard & ((sticky != 0u) | (q0 & 1u));",
     "const uint32_t up = guard;", ("muldt", "ties")),
    ("the constant multiply takes a wrong constant", "return dmul_fields(xl, xh, yl, b1, er, xh & 0x80000000u);",
     "return dmul_fields(xl, xh, yl ^ 1u, b1, er, xh & 0x80000000u);", ("mulbeta", "cipher")),
    ("dadd rounds half down", "const uint64_t T = R + ((1u << (rp - 1u)) - 1u + last);",
     "const uint64_t T = R + ((1u << (rp - 1u)) - 1u);", ("add", "ties")),
    ("dadd drops the sticky bit", "(s0 | (lost != 0u ? 1u : 0u)) ^ m", "s0 ^ m", ("sub", "gap")),
    ("the adders' shared core drops the sticky bit", "(s0 | (lost != 0u ? 1u : 0u)) ^ m", "s0 ^ m",
     ("addkick", "gap")),
    ("the known-order adder subtracts at a gap of one", "d - 1u - sub <= 30u - sub", "d - 1u <= 30u",
     ("addz", "gap1")),
    ("the known-order adder returns x + 0 = x for a zero or subnormal x",
     "&& ((xh >> 20) & 0x7FFu) - 1u <= 2045u) return x;", ") return x;", ("addkick", "zeros")),
    ("the known-order adder ignores the addend's sign", "(kAPos ? 0u : ah >> 31)", "0u", ("addz", "cipher_z")),
    ("floor truncates negatives", "return 0u - ip - (frac != 0u ? 1u : 0u);", "return 0u - ip;",
     ("floor13", "cipher")),
    ("mul_small rounds half up", "const uint32_t up = (rem > half || (rem == half && (q0 & 1u))) ? 1u : 0u;\n"
     "  q0 += up;\n  q1 += (q0 < up) ? 1u : 0u;\n  // biased exponent of the result: e + E + sh",
     "const uint32_t up = (rem >= half) ? 1u : 0u;\n"
     "  q0 += up;\n  q1 += (q0 < up) ? 1u : 0u;\n  // biased exponent of the result: e + E + sh",
     ("mul10", "cipher")),
]


@pytest.mark.parametrize("what,old,new,must_fail", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_rounding_mistakes_are_caught(tmp_path, what, old, new, must_fail):
    src = open(HEADER).read()
    assert src.count(old) == 1, what
    (tmp_path / "softfp64.cuh").write_text(src.replace(old, new))
    exe = _compile(str(tmp_path / "harness"), str(tmp_path))
    rc, rows = _run(exe, 0.05)
    assert rc == 1, what
    assert rows[must_fail]["bad"] > 0, (what, rows[must_fail])
