"""Failure behaviour: no silent CPU fallback, argument errors as status codes,
and the benchmark's reference arm on the host."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1201_3114_gb300 import lc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_missing_library_fails_loudly():
    code = ("import os, sys; sys.path.insert(0, %r)\n"
            "from paper_1201_3114_gb300 import lc\n"
            "lc.lc_version()\n" % ROOT)
    env = dict(os.environ, LC_LIBRARY="/nonexistent/liblorenzcipher.so")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True)
    assert r.returncode != 0
    assert "liblorenzcipher.so is missing" in r.stderr


def test_reference_arm_runs_on_host():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--ref-sample-mb", "1", "--messages", "64"],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_status_strings_cover_every_code():
    names = {lc.lc_status_string(s) for s in range(8)}
    assert len(names) == 8 and lc.lc_status_string(99) == "unknown status"
    assert lc.lc_last_cuda_error() == "" or isinstance(lc.lc_last_cuda_error(), str)


@pytest.mark.gpu
def test_argument_errors_are_status_codes():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with lc.Context(0) as ctx:
        h = ctx.handle
        P = torch.zeros(100, dtype=torch.uint8, device="cuda")
        Cb = torch.zeros(108, dtype=torch.uint8, device="cuda")
        assert lc.lc_encrypt(h, b"pw", None, 100, Cb, 108) == lc.LC_ERR_ARG
        assert lc.lc_encrypt(h, b"pw", P, 100, None, 108) == lc.LC_ERR_ARG
        assert lc.lc_encrypt(h, b"", P, 100, Cb, 108) == lc.LC_ERR_PASSWORD
        assert lc.lc_encrypt(h, b"x" * 33, P, 100, Cb, 108) == lc.LC_ERR_PASSWORD
        assert lc.lc_encrypt(h, b"pw", P, 100, Cb, 107) == lc.LC_ERR_LENGTH
        assert lc.lc_encrypt(h, b"pw", P, 100, P.data_ptr() + 50, 108) == lc.LC_ERR_ARG
        assert lc.lc_encrypt(h, b"pw", P, 100, Cb, 108, mode=7) == lc.LC_ERR_ARG
        assert lc.lc_encrypt(h, b"pw", P, 100, Cb, 108) == lc.LC_OK
        assert lc.lc_decrypt(h, b"pw", Cb, 7, P, 100) == lc.LC_ERR_LENGTH
        assert lc.lc_decrypt(h, b"pw", Cb, 108, P, 99) == lc.LC_ERR_LENGTH
        assert lc.lc_decrypt(h, b"pw", Cb, 108, P, 100) == lc.LC_OK
        bad = lc.params(k=(9, 4, 4))
        assert lc.lc_ctx_set_params(h, bad) == lc.LC_ERR_ARG
        bad = lc.params(block_len=100)
        assert lc.lc_ctx_set_params(h, bad) == lc.LC_ERR_ARG
        good = lc.params(dt=0.005)
        assert lc.lc_ctx_set_params(h, good) == lc.LC_OK
        assert lc.lc_ctx_get_params(h).dt == 0.005
        assert lc.lc_ctx_set_launch(h, 48) == lc.LC_ERR_ARG
        with pytest.raises(lc.LcError):
            lc.check(lc.lc_encrypt(h, b"", P, 100, Cb, 108), "lc_encrypt")
        # the pipelined host-buffer calls
        import ctypes as C
        lib = lc.load()
        hin = np.zeros(100, dtype=np.uint8)
        hout = np.zeros(108, dtype=np.uint8)
        st = np.full(1, -1, dtype=np.int32)
        b = lc.Batch([(b"pw", lc.LC_ENCRYPT, hin, 100, hout, 108)])
        assert lib.lc_submit_batch_host(h, b.reqs, 1, st.ctypes.data, 0, None, None) == lc.LC_ERR_ARG
        t = C.c_uint64(0)
        assert lib.lc_submit_batch_host(h, None, 1, st.ctypes.data, 0, None, C.byref(t)) == lc.LC_ERR_ARG
        assert lib.lc_submit_batch_host(h, b.reqs, 1, None, 0, None, C.byref(t)) == lc.LC_ERR_ARG
        assert lib.lc_submit_batch_host(h, b.reqs, 1, st.ctypes.data, 9, None, C.byref(t)) == lc.LC_ERR_ARG
        assert lc.lc_wait_batch_host(h, 0) == lc.LC_ERR_ARG
        rc, t1 = lc.lc_submit_batch_host(h, b, st)
        assert rc == lc.LC_OK and t1 > 0
        assert lc.lc_wait_batch_host(h, t1 + 1) == lc.LC_ERR_ARG
        assert lc.lc_wait_batch_host(h, t1) == lc.LC_OK and st[0] == lc.LC_OK
        # a request error is a status, not a call error
        bad = lc.Batch([(b"", lc.LC_ENCRYPT, hin, 100, hout, 108)])
        rc, t2 = lc.lc_submit_batch_host(h, bad, st)
        assert rc == lc.LC_OK and lc.lc_wait_batch_host(h, t2) == lc.LC_OK
        assert st[0] == lc.LC_ERR_PASSWORD
