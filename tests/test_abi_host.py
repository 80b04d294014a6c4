"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every symbol the header declares, and its host logic (key schedule of
Sec. 3.1, framing lengths, batch validation) agrees with the oracle."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_1201_3114_gb300 import lc, synth


def test_library_exports_every_declared_symbol():
    lib = lc.load()
    names = lc.header_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding wraps each of them under the same name
    for n in names:
        assert callable(getattr(lc, n)), n


def test_binding_constants_match_header():
    import re
    text = open(lc.HEADER).read()
    defs = dict(re.findall(r"#define\s+(LC_[A-Z0-9_]+)\s+(\d+)u?", text))
    for name in ("LC_STATS_MAX_LAG", "LC_HOST_INFLIGHT"):
        assert int(defs[name]) == getattr(lc, name), name


def test_version_and_status_strings():
    assert lc.lc_version() == 1
    for s in range(8):
        assert lc.lc_status_string(s)
    assert lc.lc_status_string(4) == "integrity check failed"


def test_default_params_match_oracle_v1():
    p = lc.lc_params_default()
    q = O.params()
    for f in ("sigma", "rho", "beta", "dt", "n_warm", "steps_per_byte", "block_len", "tag_len", "eta",
              "omega_alpha_shift", "reserved"):
        assert getattr(p, f) == getattr(q, f), f
    assert list(p.lam) == list(q.lam) and list(p.k) == list(q.k)


def _pw_cases():
    out = [b"123456", b"1234567", b"A", b"AB", b"\x00\x00\x00", b"\xff" * 32, bytes(range(1, 33))]
    for length in range(1, 33):
        for rep in range(3):
            out.append(synth.password(synth.subseed(31, 100 * length + rep), length))
    rng = np.random.default_rng(5)
    for _ in range(64):
        out.append(rng.integers(0, 256, int(rng.integers(1, 33)), dtype=np.uint8).tobytes())
    return out


def test_key_schedule_matches_oracle():
    for k in ((4, 4, 4), (3, 4, 4), (8, 5, 1)):
        pl = lc.params(k=k)
        po = O.params(k=k)
        for pw in _pw_cases():
            st, ki = lc.lc_key_info(pw, pl)
            assert st == lc.LC_OK
            ko = O.key_schedule(pw, po)
            assert list(ki.aprime) == list(ko.aprime), pw
            assert list(ki.mu) == list(ko.mu), pw
            assert list(ki.omega) == list(ko.omega), pw
            assert (ki.L, ki.D) == (ko.L, ko.D)


def test_key_schedule_rejects_bad_passwords():
    assert lc.lc_key_info(b"", None)[0] == lc.LC_ERR_PASSWORD
    assert lc.lc_key_info(b"x" * 33, None)[0] == lc.LC_ERR_PASSWORD
    assert lc.lc_key_info(b"x" * 32, None)[0] == lc.LC_OK


def test_lengths_match_oracle():
    for blen, tlen in ((4096, 8), (64, 3), (16, 1)):
        pl = lc.params(block_len=blen, tag_len=tlen)
        po = O.params(block_len=blen, tag_len=tlen)
        # lengths are a property of the parameters; use a context-free query
        # through the batch planner and the oracle's framing
        for n in list(range(0, 3 * blen + 20)) + [10 ** 6]:
            for mode in (lc.LC_PARALLEL, lc.LC_SEQUENTIAL):
                c = O.ciphertext_len(n, mode, po)
                b = lc.Batch([(b"pw", lc.LC_ENCRYPT, 0x1000, n, 0x7000_0000_0000, c)])
                rc, st, rows = lc.lc_plan_batch(b, mode, pl)
                assert rc == lc.LC_OK and st[0] == lc.LC_OK
                assert rows == O.nblocks(n, mode, po)
                b = lc.Batch([(b"pw", lc.LC_ENCRYPT, 0x1000, n, 0x7000_0000_0000, c - 1)])
                assert lc.lc_plan_batch(b, mode, pl)[1][0] == lc.LC_ERR_LENGTH
    # default-parameter context-free helpers
    for n in (0, 1, 4095, 4096, 4097, 123457):
        assert lc.lc_ciphertext_len(None, n, lc.LC_PARALLEL) == O.ciphertext_len(n, O.PARALLEL)
        c = O.ciphertext_len(n, O.PARALLEL)
        assert lc.lc_plaintext_len(None, c, lc.LC_PARALLEL) == n
    for c in range(0, 3 * 4104 + 20):
        assert lc.lc_plaintext_len(None, c, lc.LC_PARALLEL) == O.plaintext_len(c, O.PARALLEL)


def test_batch_validation():
    A = 0x1000_0000
    cases = [
        ((b"pw", 0, A, 100, A + 4096, 108), lc.LC_OK),
        ((b"pw", 0, A, 100, A + 4096, 107), lc.LC_ERR_LENGTH),
        ((b"", 0, A, 100, A + 4096, 108), lc.LC_ERR_PASSWORD),
        ((b"x" * 33, 0, A, 100, A + 4096, 108), lc.LC_ERR_PASSWORD),
        ((b"pw", 2, A, 100, A + 4096, 108), lc.LC_ERR_ARG),
        ((b"pw", 0, A, 100, A + 50, 108), lc.LC_ERR_ARG),   # partial overlap
        ((b"pw", 0, A, 100, A, 108), lc.LC_OK),             # in place
        ((b"pw", 0, None, 0, A, 8), lc.LC_OK),              # empty message
        ((b"pw", 0, None, 5, A, 13), lc.LC_ERR_ARG),
        ((b"pw", 1, A, 108, A + 4096, 100), lc.LC_OK),
        ((b"pw", 1, A, 107, A + 4096, 100), lc.LC_OK),       # n = 99 fits
        ((b"pw", 1, A, 108, A + 4096, 99), lc.LC_ERR_LENGTH),
        ((b"pw", 1, A, 7, A + 4096, 0), lc.LC_ERR_LENGTH),
        ((b"pw", 1, A, 8, None, 0), lc.LC_OK),              # empty plaintext
        ((b"pw", 1, A, 108, A + 4, 100), lc.LC_ERR_ARG),
        ((b"pw", 1, A, 4096 + 9, A + 8192, 4096), lc.LC_ERR_LENGTH),  # between valid lengths
    ]
    b = lc.Batch([c for c, _ in cases])
    rc, st, rows = lc.lc_plan_batch(b, lc.LC_PARALLEL)
    assert rc == lc.LC_OK
    assert list(st) == [want for _, want in cases]


def test_per_request_key_material_validation():
    # Sec. 3.1: -15.67 < lambda_1 < 16.01, -11.28 < lambda_2 < 16.01,
    # 0.090 < lambda_3 < 62, 2 < k_i <= 4; outside them the request fails.
    A = 0x1000_0000
    base = (b"pw", 0, A, 100, A + 4096, 108)
    cases = [
        (None, None, lc.LC_OK),
        ((1.0, 1.0, 20.0), (4, 4, 4), lc.LC_OK),
        ((-15.66, -11.27, 0.091), (3, 3, 3), lc.LC_OK),
        ((16.0, 16.0, 61.99), None, lc.LC_OK),
        (None, (3, 4, 3), lc.LC_OK),
        ((-15.67, 0.0, 20.0), None, lc.LC_ERR_ARG),
        ((0.0, 16.01, 20.0), None, lc.LC_ERR_ARG),
        ((0.0, 0.0, 0.09), None, lc.LC_ERR_ARG),
        ((0.0, 0.0, 62.0), None, lc.LC_ERR_ARG),
        ((float("nan"), 0.0, 20.0), None, lc.LC_ERR_ARG),
        (None, (2, 4, 4), lc.LC_ERR_ARG),
        (None, (4, 5, 4), lc.LC_ERR_ARG),
        (None, (4, 4, 0), lc.LC_ERR_ARG),
    ]
    b = lc.BatchEx([base + (lam, k) for lam, k, _ in cases] + [(b"", 0, A, 100, A + 4096, 108, None, (3, 3, 3))])
    rc, st, rows = lc.lc_plan_batch_ex(b, lc.LC_PARALLEL)
    assert rc == lc.LC_OK
    assert list(st) == [want for _, _, want in cases] + [lc.LC_ERR_PASSWORD]
    assert rows == sum(1 for _, _, w in cases if w == lc.LC_OK)


def test_context_needs_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lc.load().lc_ctx_create(0, C.byref(h)) == lc.LC_ERR_CUDA
    assert h.value is None


def test_splitmix64_reference_vector():
    # SplitMix64 (Steele, Lea & Flood 2014) from seed 1234567: the first
    # outputs of the published reference implementation.
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [int(x) for x in synth.words(1234567, 0, 5)] == want
    b = synth.uniform_bytes(1234567, 24)
    assert b.tobytes() == b"".join(w.to_bytes(8, "little") for w in want[:3])
    assert synth.uniform_bytes(1234567, 11, offset=5).tobytes() == b.tobytes()[5:16]


def test_workload_generators_shapes():
    c1 = synth.cfg1()
    assert c1["P"].size == 65536 and len(c1["pw"]) == 16
    assert all(32 <= ch <= 126 for ch in c1["pw"])
    c2 = synth.cfg2()
    P = c2["P"]
    assert P.size == 1 << 20 and len(c2["pw"]) == 32
    nz = P[P != 0]
    assert nz.min() >= 32 and nz.max() <= 126
    assert np.bincount(nz).argmax() == 32  # space is the most frequent symbol
    zero_runs = np.flatnonzero(P == 0)
    assert zero_runs.size == 4096 and zero_runs[-1] - zero_runs[0] == 4095
    spec = synth.cfg4_spec(count=256)
    assert spec["sizes"].min() >= 1024 and spec["sizes"].max() <= 4 << 20
    assert all(8 <= len(p) <= 32 for p in spec["pws"])
    s5 = synth.cfg5_spec(duration=1.0)
    assert 19000 < s5["t"].size < 21000
    assert abs(s5["kind"].mean() - 0.5) < 0.02
