"""The checked build (-DLC_CHECKED): its kernels validate every part-table
entry and part range before use.  The parity tests that cover batches, part
ranges, alignments and both modes run again through it, in a subprocess that
loads the checked library, and must give the same bit-exact results with no
entry reported invalid (an invalid entry makes the batch call fail)."""
import os
import subprocess
import sys

import pytest

from paper_1201_3114_gb300 import build as libbuild

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_passes_parity():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = libbuild.build(checked=True)
    env = dict(os.environ, LC_LIBRARY=lib)
    probe = subprocess.run(
        [sys.executable, "-c", "import sys; sys.path.insert(0, %r)\n"
         "from paper_1201_3114_gb300 import lc\n"
         "print(lc.lc_build_flags())" % ROOT],
        env=env, capture_output=True, text=True, timeout=300)
    assert probe.returncode == 0, probe.stderr
    assert int(probe.stdout.strip()) == 1  # the checked library is the one loaded
    sel = ("config1 or edge_sizes or every_alignment_pair or batch_mixed or in_place or "
           "config2 or tamper_every or batch_reports or submitted_host or parameter_profiles")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_gpu_parity.py"),
                        "-q", "-m", "gpu", "-k", sel, "-p", "no:cacheprovider"],
                       env=env, capture_output=True, text=True, timeout=1200, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "failed" not in r.stdout
