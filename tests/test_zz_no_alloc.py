"""lc_run_batch_noalloc: the batched path for callers that cannot allocate
device memory (memory owned by another pool, code inside an allocator
callback, threads that must not hit cudaMalloc's synchronisation).

Called through the C ABI; each result must equal, byte for byte, what the
context-based lc_run_batch produces for the same requests, on two calls in
a row (the second reuses the static scratch the first left behind), and
what the CPU oracle computes (decryption inputs are the oracle's
ciphertexts).  This file runs last so that a failure here cannot hide
another test's result; it builds all of its own inputs and also passes
alone in a fresh process.
"""
import numpy as np
import pytest

import oracle as O
from paper_1201_3114_gb300 import lc, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
B = 4096


def _requests(mode, seed):
    """A mixed batch: both directions, empty / ragged / multi-part messages,
    one tampered ciphertext, one request that fails validation.  Returns the
    plan, the device inputs and the oracle's expected output per request."""
    rng = np.random.default_rng(seed)
    sizes = [0, 1, 15, 16, 17, B - 1, B, B + 1, 3 * B + 5, 40000, 123457, 5]
    keep, plan, expect = [], [], []
    for i, n in enumerate(sizes):
        pw = synth.password(synth.subseed(seed, i), 1 + (3 * i) % 32)
        P = synth.uniform_bytes(synth.subseed(seed + 1, i), n)
        ct = O.encrypt(pw, P, mode)
        d = i % 2
        if d == 0:
            src, want = P, ct
        else:
            src, want = ct.copy(), P
            if i == 9:  # tampered: must be rejected and zeroed
                src[int(rng.integers(0, src.size))] ^= 0x5A
                want = np.zeros(n, dtype=np.uint8)
        dsrc = torch.from_numpy(np.ascontiguousarray(src)).cuda()
        keep.append(dsrc)
        plan.append((pw, d, dsrc, src.size, want.size))
        expect.append(want)
    plan.append((b"", 0, keep[0], 0, 8))  # empty password: validation error
    expect.append(None)
    torch.cuda.synchronize()
    return plan, keep, expect


def _run(entry, plan, mode, ctx=None):
    outs = [torch.full((max(1, o),), 0xEE, dtype=torch.uint8, device="cuda") for *_, o in plan]
    items = [(pw, d, src if ln else None, ln, out, o) for (pw, d, src, ln, o), out in zip(plan, outs)]
    status = torch.full((len(items),), -1, dtype=torch.int32, device="cuda")
    b = lc.Batch(items)
    if entry == "ctx":
        rc = lc.lc_run_batch(ctx.handle, b, status, mode)
    else:
        rc = lc.lc_run_batch_noalloc(b, status, mode)
    assert rc == lc.LC_OK
    torch.cuda.synchronize()
    return status.cpu().numpy(), [o.cpu().numpy()[:max(0, p[4])] for o, p in zip(outs, plan)]


@pytest.mark.parametrize("mode", [lc.LC_PARALLEL, lc.LC_SEQUENTIAL])
def test_noalloc_matches_run_batch_twice(mode):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    plan, keep, expect = _requests(mode, 900 + mode)
    with lc.Context(0) as ctx:
        want_st, want_out = _run("ctx", plan, mode, ctx)
    assert want_st[-1] == lc.LC_ERR_PASSWORD
    assert want_st[9] == lc.LC_ERR_INTEGRITY
    assert all(s == lc.LC_OK for k, s in enumerate(want_st[:-1]) if k != 9)
    for call in range(2):
        st, out = _run("noalloc", plan, mode)
        assert list(st) == list(want_st), call
        for k, (a, b) in enumerate(zip(out, want_out)):
            assert np.array_equal(a, b), (call, k)
            # and the oracle's bytes (validation failures have none)
            if expect[k] is not None:
                assert np.array_equal(a, expect[k]), (call, k)


def test_noalloc_allocates_nothing_and_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    plan, keep, _ = _requests(lc.LC_PARALLEL, 950)
    _run("noalloc", plan, lc.LC_PARALLEL)  # first call on the device sets it up
    outs = [torch.zeros(max(1, o), dtype=torch.uint8, device="cuda") for *_, o in plan]
    items = [(pw, d, src if ln else None, ln, out, o) for (pw, d, src, ln, o), out in zip(plan, outs)]
    status = torch.zeros(len(items), dtype=torch.int32, device="cuda")
    b = lc.Batch(items)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert lc.lc_run_batch_noalloc(b, status, lc.LC_PARALLEL) == lc.LC_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # Beyond the fixed capacity: rejected on the host before any GPU work.
    too_many = lc.Batch([(b"pw", 0, None, 0, outs[0], 8)] * 1025)
    st = torch.zeros(1025, dtype=torch.int32, device="cuda")
    assert lc.lc_run_batch_noalloc(too_many, st, lc.LC_PARALLEL) == lc.LC_ERR_LENGTH
    big_n = 240001 * B
    src = torch.zeros(big_n, dtype=torch.uint8, device="cuda")
    dst = torch.zeros(big_n + 8 * 240001, dtype=torch.uint8, device="cuda")
    too_big = lc.Batch([(b"pw", 0, src, big_n, dst, dst.numel())])
    assert lc.lc_run_batch_noalloc(too_big, st, lc.LC_PARALLEL) == lc.LC_ERR_LENGTH
    torch.cuda.synchronize()
    assert int(dst[:1 << 20].sum()) == 0  # nothing ran
