"""Planted mistakes in copies of the oracle must fail its pins.

Each case below copies oracle/lco.c, plants one plausible misreading of the
paper (a dropped term, a wrong index, a wrong order of sub-steps, an
off-by-one count), compiles the copy with the oracle's own flags and runs
the oracle's pin suites (test_oracle_steps.py, then test_oracle_pins.py)
against it in a subprocess.  The pins are shown to bite: every copy must
make at least one of them fail, while the unmodified source passes them.
The cases cover Sec. 3.2 Steps 2 and 3 (r_i = F[r_{i-1} + M(P_i)] of
Sec. 2), the warm-up (n_it, Sec. 3.1), Eq. 6 for alpha, reading R16 for
decryption, the part offset of Sec. 5 and the tag plaintext LE64(n).
"""
import os
import shutil
import subprocess
import sys

import pytest

from oracle import build as obuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lco.c")
HDR = os.path.join(ROOT, "oracle", "lco.h")
PIN_FILES = ["tests/test_oracle_steps.py", "tests/test_oracle_pins.py"]

KICK = "  st->r[st->mu[2]] = st->r[st->mu[2]] + theta;\n"
EULER = "  for (s = 0; s < p->steps_per_byte; s++) lco_euler_step(p, st->r);\n"
MU = ("  for (i = 0; i < 3; i++)\n"
      "    st->mu[i] = (st->mu[i] + lco_rbyte(st->alpha[i], st->omega[i])) % 3u;\n")
ALPHA = "  for (i = 0; i < 3; i++) st->alpha[i] = st->r[st->mu[i]];\n"
OMEGA = ("  for (i = 0; i < 3; i++)\n"
         "    st->omega[i] = (st->omega[i] + lco_rbyte(st->alpha[p->omega_alpha_shift ? (i + 2) % 3 : i],\n"
         "                                             st->omega[i])) % p->k[i];\n")
APRIME = "  for (i = 0; i < 3; i++) st->r[i] = st->r[i] + K->aprime[i];\n"
WARM = "  for (s = 0; s < p->n_warm; s++) lco_euler_step(p, st->r);\n"
START_COPY = ("  for (j = 0; j < 3; j++) {\n    st->mu[j] = K->mu[j];\n"
              "    st->omega[j] = K->omega[j];\n    st->alpha[j] = st->r[st->mu[j]];\n  }\n")

MUTANTS = [
    # (name, text replaced, replacement)
    ("no r += a' at the end of Step 3", APRIME, ""),
    ("kick on r[mu_1] instead of r[mu_3]", KICK,
     "  st->r[st->mu[0]] = st->r[st->mu[0]] + theta;\n"),
    ("F before the kick", KICK + EULER, EULER + KICK),
    ("n_warm - 1 warm-up steps", WARM,
     "  for (s = 1; s < p->n_warm; s++) lco_euler_step(p, st->r);\n"),
    ("n_warm + 1 warm-up steps", WARM,
     "  for (s = 0; s <= p->n_warm; s++) lco_euler_step(p, st->r);\n"),
    ("old alpha in the Omega update", ALPHA + OMEGA, OMEGA + ALPHA),
    ("alpha re-read with the old mu", MU + ALPHA, ALPHA + MU),
    ("mu moved with the new Omega", MU + ALPHA + OMEGA, OMEGA + MU + ALPHA),
    ("r += a' before F", KICK + EULER, KICK + APRIME + EULER),
    ("Theta divides by 10^(3 + Omega_1)", "theta = (double)P / TEN[3 + st->omega[2]];",
     "theta = (double)P / TEN[3 + st->omega[0]];"),
    ("decryption kicks with the ciphertext byte", "    P = y; /* reading R16",
     "    P = x; /* reading R16"),
    ("alpha sampled before the warm-up", WARM + START_COPY, START_COPY + WARM),
    ("part offset on x only", "st->r[j] = (K->aprime[j] + p->lambda[j]) + (double)b * p->eta;",
     "st->r[j] = (K->aprime[j] + p->lambda[j]) + (j == 0 ? (double)b * p->eta : 0.0);"),
    ("tag plaintext big-endian", "return (uint32_t)(((uint64_t)n >> (8 * t)) & 255u);",
     "return (uint32_t)(((uint64_t)n >> (8 * (7 - t))) & 255u);"),
]


def _compile(src_text, out_dir):
    if shutil.which("gcc") is None:
        pytest.skip("no host C compiler")
    os.makedirs(out_dir, exist_ok=True)
    c = os.path.join(out_dir, "lco.c")
    with open(c, "w") as f:
        f.write(src_text)
    shutil.copy(HDR, os.path.join(out_dir, "lco.h"))
    lib = os.path.join(out_dir, "liblco.so")
    subprocess.run(["gcc"] + obuild.CFLAGS + ["-o", lib, c, "-lm"], check=True, capture_output=True,
                   text=True)
    return lib


def _run_pins(lib):
    env = dict(os.environ, LCO_LIBRARY=lib)
    p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m",
                        "not gpu"] + PIN_FILES, cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    failed = [ln.split()[1] for ln in p.stdout.splitlines() if ln.startswith("FAILED ")]
    return p.returncode, failed, p.stdout[-2000:]


def test_unmodified_oracle_passes_the_pins(tmp_path):
    with open(SRC) as f:
        lib = _compile(f.read(), str(tmp_path / "control"))
    rc, failed, tail = _run_pins(lib)
    assert rc == 0 and not failed, tail


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new):
    with open(SRC) as f:
        src = f.read()
    assert src.count(old) == 1, "planted text not found exactly once: " + name
    mutated = src.replace(old, new)
    assert mutated != src
    lib = _compile(mutated, str(tmp_path / "mutant"))
    rc, failed, tail = _run_pins(lib)
    # exit status 1: tests ran and at least one failed (not a crash or a
    # collection error)
    assert rc == 1 and failed, (name, rc, tail)
