"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Every comparison is bit-exact (tolerance 0): the outputs are bytes and
verdicts, and the trajectory arithmetic is required to round exactly as
the oracle does.  Inputs are seeded and synthetic (paper_1201_3114_gb300.synth).
"""
import numpy as np
import pytest

import oracle as O
import oracle_mt
from paper_1201_3114_gb300 import lc, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
B = 4096
T = 8


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = lc.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def gpu_encrypt(ctx, pw, P, mode=lc.LC_PARALLEL):
    return host(ctx.encrypt(pw, dev(P), mode))


def gpu_decrypt(ctx, pw, Cb, mode=lc.LC_PARALLEL):
    st, out = ctx.decrypt(pw, dev(Cb), mode)
    return st, host(out)


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------

def test_device_generator_matches_host():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    for seed in (1234567, synth.config_seed(3)):
        for off in (0, 1, 3, 8, 13, 4096 * 7 + 5):
            for n in (1, 7, 8, 9, 100, 4096, 65536 + 3):
                buf = torch.empty(n + 16, dtype=torch.uint8, device="cuda")
                for shift in (0, 3):
                    lc.check(lc.lc_synth_uniform(buf[shift:].data_ptr(), n, seed, off))
                    got = host(buf)[shift:shift + n]
                    assert np.array_equal(got, synth.uniform_bytes(seed, n, off)), (seed, off, n, shift)


# ---------------------------------------------------------------------------
# single messages
# ---------------------------------------------------------------------------

def test_config1_64k(ctx):
    c = synth.cfg1()
    want = O.encrypt(c["pw"], c["P"], O.PARALLEL)
    got = gpu_encrypt(ctx, c["pw"], c["P"])
    assert np.array_equal(got, want)
    st, back = gpu_decrypt(ctx, c["pw"], got)
    assert st == lc.LC_OK and np.array_equal(back, c["P"])


SIZES = [0, 1, 2, 15, 16, 17, 31, 33, 255, B - 1, B, B + 1, B + 16, 2 * B - 3, 3 * B + 5]


@pytest.mark.parametrize("mode", [lc.LC_PARALLEL, lc.LC_SEQUENTIAL])
def test_edge_sizes(ctx, mode):
    for i, n in enumerate(SIZES):
        pw = synth.password(synth.subseed(40, i), 1 + (5 * i) % 32)
        P = synth.uniform_bytes(synth.subseed(41, i), n)
        want = O.encrypt(pw, P, mode)
        got = gpu_encrypt(ctx, pw, P, mode)
        assert np.array_equal(got, want), (n, mode)
        st, back = gpu_decrypt(ctx, pw, got, mode)
        assert st == lc.LC_OK and np.array_equal(back, P), (n, mode)


def test_every_password_length(ctx):
    P = synth.uniform_bytes(42, 3 * B + 77)
    for length in range(1, 33):
        pw = synth.password(synth.subseed(43, length), length)
        assert np.array_equal(gpu_encrypt(ctx, pw, P), O.encrypt(pw, P)), length
    for pw in (b"\x00\x00\x00", b"\xff" * 32, b"\x80"):
        assert np.array_equal(gpu_encrypt(ctx, pw, P), O.encrypt(pw, P)), pw


def test_unaligned_buffers(ctx):
    # Misaligned input or output pointers; results agree.
    n = 2 * B + 21
    P = synth.uniform_bytes(44, n)
    pw = b"unaligned-buffers"
    want = O.encrypt(pw, P)
    for pin, pout in ((1, 0), (0, 3), (5, 7), (16, 16)):
        src = torch.zeros(n + 64, dtype=torch.uint8, device="cuda")
        dst = torch.zeros(want.size + 64, dtype=torch.uint8, device="cuda")
        src[pin:pin + n] = dev(P)
        st = lc.lc_encrypt(ctx.handle, pw, src.data_ptr() + pin, n, dst.data_ptr() + pout,
                           want.size, lc.LC_PARALLEL)
        assert st == lc.LC_OK
        got = host(dst)[pout:pout + want.size]
        assert np.array_equal(got, want), (pin, pout)
        back = torch.zeros(n + 64, dtype=torch.uint8, device="cuda")
        st = lc.lc_decrypt(ctx.handle, pw, dst.data_ptr() + pout, want.size, back.data_ptr() + pin,
                           n, lc.LC_PARALLEL)
        assert st == lc.LC_OK and np.array_equal(host(back)[pin:pin + n], P)


@pytest.mark.parametrize("mode", [lc.LC_PARALLEL, lc.LC_SEQUENTIAL])
def test_every_alignment_pair(ctx, mode):
    # Every (source, destination) offset modulo 16, both directions, in one
    # batch: head bytes, the realigned 16-byte body and the tail all vary.
    reqs, want_out, outs = [], [], []
    keep = []
    k = 0
    for pin in range(16):
        for pout in range(16):
            n = B + 37 + (k % 23) if mode == lc.LC_PARALLEL else 300 + k % 41
            pw = synth.password(synth.subseed(46, k), 1 + k % 32)
            P = synth.uniform_bytes(synth.subseed(47, k), n)
            Cw = O.encrypt(pw, P, mode)
            for d, x, y in ((0, P, Cw), (1, Cw, P)):
                src = torch.zeros(x.size + 32, dtype=torch.uint8, device="cuda")
                dst = torch.full((y.size + 32,), 0x5A, dtype=torch.uint8, device="cuda")
                src[pin:pin + x.size] = dev(x)
                reqs.append((pw, d, src.data_ptr() + pin, x.size, dst.data_ptr() + pout, y.size))
                want_out.append((pout, y))
                outs.append(dst)
                keep.append(src)
            k += 1
    st = torch.full((len(reqs),), -1, dtype=torch.int32, device="cuda")
    lc.check(lc.lc_run_batch(ctx.handle, lc.Batch(reqs), st, mode))
    assert (host(st) == 0).all()
    for i, ((pout, y), dst) in enumerate(zip(want_out, outs)):
        got = host(dst)
        assert np.array_equal(got[pout:pout + y.size], y), i
        assert (got[:pout] == 0x5A).all() and (got[pout + y.size:] == 0x5A).all(), i


@pytest.mark.parametrize("shape", [(256, 0, 0, 0), (256, 0, 0, 0, 0, 0, 0, 1), (256, 0, 0, 1)],
                         ids=["three-warps", "fp64-only", "int-split"])
def test_in_place(ctx, shape):
    # every build reads each byte before it is written
    n = 3 * B + 9
    P = synth.uniform_bytes(45, n)
    pw = b"in-place"
    want = O.encrypt(pw, P)
    buf = torch.zeros(want.size, dtype=torch.uint8, device="cuda")
    buf[:n] = dev(P)
    try:
        assert lc.lc_ctx_set_launch(ctx.handle, *shape) == lc.LC_OK
        for mode in (lc.LC_PARALLEL, lc.LC_SEQUENTIAL):
            want = O.encrypt(pw, P, mode)
            buf = torch.zeros(want.size, dtype=torch.uint8, device="cuda")
            buf[:n] = dev(P)
            assert lc.lc_encrypt(ctx.handle, pw, buf, n, buf, want.size, mode) == lc.LC_OK
            assert np.array_equal(host(buf), want), mode
            assert lc.lc_decrypt(ctx.handle, pw, buf, want.size, buf, n, mode) == lc.LC_OK
            assert np.array_equal(host(buf)[:n], P), mode
    finally:
        lc.lc_ctx_set_launch(ctx.handle, 256, 0)


def test_config2_text_both_modes_and_tamper(ctx):
    c = synth.cfg2()
    P, pw = c["P"], c["pw"]
    for mode in (lc.LC_PARALLEL, lc.LC_SEQUENTIAL):
        want = O.encrypt(pw, P, mode)
        got = gpu_encrypt(ctx, pw, P, mode)
        assert np.array_equal(got, want), mode
        st, back = gpu_decrypt(ctx, pw, got, mode)
        assert st == lc.LC_OK and np.array_equal(back, P)
        # the flipped copy is made from the oracle's ciphertext (equal to the
        # GPU's, as checked above), so the oracle never reads a GPU output
        pos = synth.word(c["flip_seed"], mode) % want.size
        bad = want.copy()
        bad[pos] ^= 1 + synth.word(c["flip_seed"], 10 + mode) % 255
        st, out = gpu_decrypt(ctx, pw, bad, mode)
        assert st == lc.LC_ERR_INTEGRITY and not out.any()
        ost, oout = O.decrypt(pw, bad, mode)
        assert ost == O.ERR_INTEGRITY


def test_wrong_password_rejected(ctx):
    P = synth.uniform_bytes(46, 5 * B)
    ct = gpu_encrypt(ctx, "123456", P)
    st, out = gpu_decrypt(ctx, "123457", ct)
    assert st == lc.LC_ERR_INTEGRITY and not out.any()


def test_tamper_every_tag_byte_and_random_body_bytes(ctx):
    # One batch decrypts many tampered copies; each must be rejected, the
    # untouched copy accepted, exactly as the oracle decides.
    pw = b"tamper"
    n = 2 * B + 50
    P = synth.uniform_bytes(47, n)
    ct = O.encrypt(pw, P)
    rng = np.random.default_rng(48)
    positions = list(range(n, ct.size)) + [int(x) for x in rng.integers(0, n, 300)]
    copies = np.tile(ct, (len(positions) + 1, 1))
    for k, pos in enumerate(positions):
        copies[k, pos] ^= int(rng.integers(1, 256))
    cin = dev(copies)
    pout = torch.zeros((len(positions) + 1, n), dtype=torch.uint8, device="cuda")
    items = [(pw, lc.LC_DECRYPT, cin[k], ct.size, pout[k], n) for k in range(len(positions) + 1)]
    status = torch.full((len(items),), -1, dtype=torch.int32, device="cuda")
    b = lc.Batch(items)
    lc.check(lc.lc_run_batch(ctx.handle, b, status))
    st = host(status)
    outs = host(pout)
    assert all(s == lc.LC_ERR_INTEGRITY for s in st[:-1])
    assert st[-1] == lc.LC_OK and np.array_equal(outs[-1], P)
    assert not outs[:-1].any()


# ---------------------------------------------------------------------------
# other parameter profiles (general-k path, several Euler steps per byte,
# divergent dt, small parts)
# ---------------------------------------------------------------------------

PROFILES = [
    dict(dt=0.027),                      # leaves the basin: NaN/inf saturation
    dict(k=(3, 4, 4)),                   # general Omega path
    dict(k=(8, 5, 1)),
    dict(steps_per_byte=3),
    dict(n_warm=0),
    dict(block_len=64, tag_len=3),
    dict(lam=(-15.0, -11.0, 61.0), eta=2.0 ** -10),
    dict(sigma=0.0, rho=0.0, beta=0.0, dt=0.0, lam=(1.5, 1.5, 1.5)),
    dict(omega_alpha_shift=1),           # Step 3's alpha index read with 0-based i
    dict(omega_alpha_shift=1, k=(3, 4, 3)),
]


@pytest.mark.parametrize("over", PROFILES, ids=lambda d: ",".join(d))
def test_parameter_profiles(over):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    po = O.params(**over)
    pl = lc.params(**over)
    with lc.Context(0, pl) as c:
        for i, n in enumerate([0, 1, 17, 63, 64, 65, 2 * B + 3]):
            for mode in (lc.LC_PARALLEL, lc.LC_SEQUENTIAL):
                pw = synth.password(synth.subseed(49, i), 3 + i)
                P = synth.uniform_bytes(synth.subseed(50, i), n)
                want = O.encrypt(pw, P, mode, po)
                got = gpu_encrypt(c, pw, P, mode)
                assert np.array_equal(got, want), (over, n, mode)
                st, back = gpu_decrypt(c, pw, got, mode)
                assert st == lc.LC_OK and np.array_equal(back, P)


# ---------------------------------------------------------------------------
# batched path
# ---------------------------------------------------------------------------

def _mixed_batch(count, seed, max_size=40000):
    rng = np.random.default_rng(seed)
    msgs = []
    for m in range(count):
        n = int(rng.choice([0, 1, 15, 16, int(rng.integers(1, max_size)), B, B + 1]))
        pw = synth.password(synth.subseed(seed, m), int(rng.integers(1, 33)))
        P = synth.uniform_bytes(synth.subseed(seed + 1, m), n)
        d = int(rng.integers(0, 2))
        msgs.append((pw, d, P))
    return msgs


@pytest.mark.parametrize("mode", [lc.LC_PARALLEL, lc.LC_SEQUENTIAL])
def test_batch_mixed_matches_oracle_and_alone(ctx, mode):
    msgs = _mixed_batch(96, 51)
    items, expect, keep = [], [], []
    for pw, d, P in msgs:
        ct = O.encrypt(pw, P, mode)
        if d == lc.LC_ENCRYPT:
            src, want = dev(P), ct
        else:
            src, want = dev(ct), P
        out = torch.zeros(max(1, want.size), dtype=torch.uint8, device="cuda")
        keep += [src, out]
        items.append((pw, d, src, src.numel() if (d or P.size) else 0, out, want.size))
        expect.append(want)
    status = torch.full((len(items),), -1, dtype=torch.int32, device="cuda")
    lc.check(lc.lc_run_batch(ctx.handle, lc.Batch(items), status, mode))
    st = host(status)
    assert all(s == lc.LC_OK for s in st)
    for k, want in enumerate(expect):
        got = host(items[k][4])[:want.size]
        assert np.array_equal(got, want), k
    # each message alone gives the same bytes as in the mix
    for k in range(0, len(items), 7):
        pw, d, src, ln, _, cap = items[k]
        out = torch.zeros(max(1, cap), dtype=torch.uint8, device="cuda")
        s1 = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        lc.check(lc.lc_run_batch(ctx.handle, lc.Batch([(pw, d, src, ln, out, cap)]), s1, mode))
        assert host(s1)[0] == lc.LC_OK
        assert np.array_equal(host(out)[:cap], expect[k])


def test_batch_reports_per_request_errors(ctx):
    P = synth.uniform_bytes(52, 1000)
    pw = b"per-request"
    ct = O.encrypt(pw, P)
    src = dev(P)
    csrc = dev(ct)
    o1 = torch.zeros(ct.size, dtype=torch.uint8, device="cuda")
    o2 = torch.zeros(ct.size, dtype=torch.uint8, device="cuda")
    o3 = torch.zeros(P.size, dtype=torch.uint8, device="cuda")
    bad = ct.copy()
    bad[3] ^= 9
    bsrc = dev(bad)
    o4 = torch.ones(P.size, dtype=torch.uint8, device="cuda")
    items = [
        (pw, 0, src, P.size, o1, ct.size),          # ok
        (b"", 0, src, P.size, o2, ct.size),         # bad password
        (pw, 0, src, P.size, o2, ct.size - 1),      # too small
        (pw, 1, csrc, ct.size, o3, P.size),         # ok
        (pw, 1, bsrc, ct.size, o4, P.size),         # tampered
        (pw, 1, csrc, T - 1, o3, P.size),           # shorter than one tag
    ]
    status = torch.full((len(items),), -1, dtype=torch.int32, device="cuda")
    lc.check(lc.lc_run_batch(ctx.handle, lc.Batch(items), status))
    assert list(host(status)) == [0, lc.LC_ERR_PASSWORD, lc.LC_ERR_LENGTH, 0, lc.LC_ERR_INTEGRITY,
                                  lc.LC_ERR_LENGTH]
    assert np.array_equal(host(o1), ct)
    assert np.array_equal(host(o3), P)
    assert not host(o4).any()


def test_host_buffer_batch_equals_device_batch(ctx):
    msgs = _mixed_batch(40, 53, max_size=20000)
    # pack every input and output contiguously in pinned host memory
    ins, outs = [], []
    for pw, d, P in msgs:
        ct = O.encrypt(pw, P)
        ins.append(P if d == 0 else ct)
        outs.append(ct if d == 0 else P)
    hin = torch.empty(sum(x.size for x in ins), dtype=torch.uint8).pin_memory()
    hout = torch.zeros(sum(x.size for x in outs), dtype=torch.uint8).pin_memory()
    items, a, b_ = [], 0, 0
    for (pw, d, _), x, y in zip(msgs, ins, outs):
        hin[a:a + x.size] = torch.from_numpy(x)
        items.append((pw, d, hin.data_ptr() + a, x.size, hout.data_ptr() + b_, y.size))
        a += x.size
        b_ += y.size
    st = np.full(len(items), -1, dtype=np.int32)
    lc.check(lc.lc_run_batch_host(ctx.handle, lc.Batch(items), st))
    assert all(s == lc.LC_OK for s in st)
    got = hout.numpy()
    b_ = 0
    for y in outs:
        assert np.array_equal(got[b_:b_ + y.size], y)
        b_ += y.size


def test_launch_shapes_do_not_change_results(ctx):
    n = 40 * B + 11
    P = synth.uniform_bytes(54, n)
    pw = b"launch-shapes"
    want = O.encrypt(pw, P)
    try:
        for tpc, cps in ((32, 1), (64, 0), (128, 2), (256, 0), (256, 4)):
            # integer-split variant (full-grid and partial-grid builds, each
            # default and dense), FP64-only variant
            for small, dense, full, split in ((1, 0, 1, 0), (1, 1, 1, 0), (1, 0, 0, 0), (1, 1, 0, 0),
                                              (0xFFFFFFFF, 0, 0, 1), (0xFFFFFFFF, 0, 0, 0xFFFFFFFF)):
                assert lc.lc_ctx_set_launch(ctx.handle, tpc, cps, 0, small, 0, dense, full, split) == lc.LC_OK
                assert np.array_equal(gpu_encrypt(ctx, pw, P), want), (tpc, cps, small, dense, full, split)
        assert lc.lc_ctx_set_launch(ctx.handle, 256, 0, 1, 0) == lc.LC_ERR_ARG
        assert lc.lc_ctx_set_launch(ctx.handle, 256, 0, 0, 0, 0, 2) == lc.LC_ERR_ARG
        best = lc.lc_tune(ctx.handle, 8 << 20)
        rep = lc.lc_tune_report(ctx.handle)
        # 3 CTA widths x (all resident / one fewer) x 2 builds, each timed
        assert 6 <= len(rep) <= 12 and all(ms > 0 for _, ms in rep)
        assert {l["dense_build"] for l, _ in rep} == {0, 1}
        fastest = min(rep, key=lambda e: e[1])[0]
        assert (best.threads_per_cta, best.ctas_per_sm, best.dense_build) == \
            (fastest["threads_per_cta"], fastest["ctas_per_sm"], fastest["dense_build"])
        assert np.array_equal(gpu_encrypt(ctx, pw, P), want)
    finally:
        lc.lc_ctx_set_launch(ctx.handle, 256, 0)


@pytest.mark.parametrize("small,full,split", [(1, 1, 0), (1, 0, 0), (0xFFFFFFFF, 0, 1),
                                              (0xFFFFFFFF, 0, 0xFFFFFFFF)],
                         ids=["int-split-full-grid", "int-split-partial-grid", "fp64-only",
                              "fp64-three-warps"])
def test_both_v1_kernel_variants(ctx, small, full, split):
    # The batched kernel has four v1 builds: binary64 multiplies (and, on a
    # full grid, the kick) on the integer pipes; everything on the FP64 pipe,
    # one part per thread or each part's coordinates on three warps; force
    # each one.
    try:
        assert lc.lc_ctx_set_launch(ctx.handle, 256, 0, 0, small, 0, 0, full, split) == lc.LC_OK
        for i, n in enumerate([0, 1, 17, B - 1, B + 1, 5 * B + 3]):
            for mode in (lc.LC_PARALLEL, lc.LC_SEQUENTIAL):
                pw = synth.password(synth.subseed(60, i), 2 + 5 * i)
                P = synth.uniform_bytes(synth.subseed(61, i), n)
                want = O.encrypt(pw, P, mode)
                got = gpu_encrypt(ctx, pw, P, mode)
                assert np.array_equal(got, want), (small, n, mode)
                st, back = gpu_decrypt(ctx, pw, got, mode)
                assert st == lc.LC_OK and np.array_equal(back, P)
        msgs = _mixed_batch(64, 62)
        items, expect = [], []
        for pw, d, P in msgs:
            ct = O.encrypt(pw, P)
            src = dev(P if d == 0 else ct)
            want = ct if d == 0 else P
            out = torch.zeros(max(1, want.size), dtype=torch.uint8, device="cuda")
            items.append((pw, d, src, src.numel(), out, want.size))
            expect.append(want)
        status = torch.full((len(items),), -1, dtype=torch.int32, device="cuda")
        lc.check(lc.lc_run_batch(ctx.handle, lc.Batch(items), status))
        assert (host(status) == 0).all()
        for k, want in enumerate(expect):
            assert np.array_equal(host(items[k][4])[:want.size], want), k
    finally:
        lc.lc_ctx_set_launch(ctx.handle, 256, 0)


def test_timing_and_launch_counters(ctx):
    P = dev(synth.uniform_bytes(55, 8 * B))
    lc.check(lc.lc_ctx_timing(ctx.handle, True))
    before = lc.lc_ctx_launch_count(ctx.handle)
    for _ in range(3):
        ctx.encrypt(b"timing", P)
    ms, n = lc.lc_ctx_kernel_time(ctx.handle)
    assert n == 3 and ms > 0
    assert lc.lc_ctx_launch_count(ctx.handle) - before == 6
    lc.check(lc.lc_ctx_timing(ctx.handle, False))


# ---------------------------------------------------------------------------
# full-size workloads, every output byte against the oracle on all host cores
# ---------------------------------------------------------------------------

def test_config3_1gib_complete(ctx):
    # 1 GiB of uniform bytes, 262,144 parts: every ciphertext byte and every
    # tag against the oracle; the oracle's ciphertext decrypts to P.
    spec = synth.cfg3_spec()
    n, pw, seed = spec["n"], spec["pw"], spec["data_seed"]
    P = oracle_mt.uniform(seed, n)
    want = oracle_mt.encrypt(pw, P)
    Pd = torch.from_numpy(P).cuda()
    try:
        # the default launch shape, then the dense build the autotuner
        # usually picks for the benchmark
        for shape in ((256, 0, 0, 0, 0, 0), (64, 0, 0, 0, 0, 1)):
            assert lc.lc_ctx_set_launch(ctx.handle, *shape) == lc.LC_OK
            got = host(ctx.encrypt(pw, Pd))
            assert got.size == want.size == n + T * (n // B)
            assert oracle_mt.first_difference(got, want) == -1, shape
            del got
    finally:
        lc.lc_ctx_set_launch(ctx.handle, 256, 0)
    st, back = ctx.decrypt(pw, torch.from_numpy(want).cuda())
    assert st == lc.LC_OK
    assert torch.equal(back, Pd)


def test_config4_batch_complete(ctx):
    # The batched workload: 4096 messages (log-uniform 1 KiB - 4 MiB, 2.06 GB),
    # the first half encrypted, the second half decrypted from ciphertexts the
    # oracle made; one launch; every output byte and every status.
    spec = synth.cfg4_spec()
    sizes, pws, seeds, dirs = spec["sizes"], spec["pws"], spec["data_seeds"], spec["dirs"]
    count = len(sizes)
    plains = oracle_mt.uniform_many(seeds, sizes)
    cts = oracle_mt.encrypt_many(list(zip(pws, plains)))
    ins = [plains[m] if dirs[m] == 0 else cts[m] for m in range(count)]
    want = [cts[m] if dirs[m] == 0 else plains[m] for m in range(count)]

    def pack(arrs):
        offs, tot = [], 0
        for a in arrs:
            offs.append(tot)
            tot = (tot + a.size + 255) & ~255
        buf = np.zeros(tot, dtype=np.uint8)
        for a, o in zip(arrs, offs):
            buf[o:o + a.size] = a
        return buf, offs

    hin, in_off = pack(ins)
    _, out_off = pack(want)
    din = torch.from_numpy(hin).cuda()
    dout = torch.full((out_off[-1] + want[-1].size + 256,), 0xA5, dtype=torch.uint8, device="cuda")
    items = [(pws[m], dirs[m], din.data_ptr() + in_off[m], ins[m].size, dout.data_ptr() + out_off[m],
              want[m].size) for m in range(count)]
    batch = lc.Batch(items)
    try:
        # the default launch shape, and the one the benchmark times: the
        # autotuner's choice on a probe of this batch's size
        for tune in (False, True):
            lc.lc_ctx_set_launch(ctx.handle, 256, 0)
            if tune:
                lc.lc_tune(ctx.handle, int(sizes.sum()))
            dout.fill_(0xA5)
            status = torch.full((count,), -1, dtype=torch.int32, device="cuda")
            lc.check(lc.lc_run_batch(ctx.handle, batch, status))
            assert (host(status) == 0).all()
            hout = host(dout)
            bad = [m for m in range(count)
                   if not np.array_equal(hout[out_off[m]:out_off[m] + want[m].size], want[m])]
            assert not bad, (tune, lc.lc_ctx_get_launch(ctx.handle).as_dict(), bad[:10])
    finally:
        lc.lc_ctx_set_launch(ctx.handle, 256, 0)


def test_n_it_steps_per_byte_profile():
    # The alternative reading of n_it: 3000 Euler steps per byte (Sec. 3.1).
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    po = O.params(steps_per_byte=3000)
    pl = lc.params(steps_per_byte=3000)
    with lc.Context(0, pl) as c:
        for i, n in enumerate([0, 1, 33, 100]):
            pw = synth.password(synth.subseed(58, i), 8 + i)
            P = synth.uniform_bytes(synth.subseed(59, i), n)
            want = O.encrypt(pw, P, O.PARALLEL, po)
            got = gpu_encrypt(c, pw, P)
            assert np.array_equal(got, want), n
            st, back = gpu_decrypt(c, pw, got)
            assert st == lc.LC_OK and np.array_equal(back, P)


def test_host_buffer_batch_pageable_and_scattered(ctx):
    # Pageable numpy buffers (one per request, not contiguous) and
    # page-locked ones both equal the oracle.
    msgs = _mixed_batch(24, 63, max_size=20000)
    ins, outs, want = [], [], []
    for pw, d, P in msgs:
        ct = O.encrypt(pw, P)
        ins.append(np.ascontiguousarray(P if d == 0 else ct))
        want.append(ct if d == 0 else P)
        outs.append(np.zeros(max(1, want[-1].size), dtype=np.uint8))
    items = [(pw, d, x, x.size, y, w.size) for (pw, d, _), x, y, w in zip(msgs, ins, outs, want)]
    st = np.full(len(items), -1, dtype=np.int32)
    lc.check(lc.lc_run_batch_host(ctx.handle, lc.Batch(items), st))
    assert (st == 0).all()
    for y, w in zip(outs, want):
        assert np.array_equal(y[:w.size], w)
    # the same requests from page-locked buffers, a tampered one among them
    pins = [torch.from_numpy(x.copy()).pin_memory() for x in ins]
    pouts = [torch.zeros(max(1, w.size), dtype=torch.uint8).pin_memory() for w in want]
    k = next(i for i, (_, d, P) in enumerate(msgs) if d == 1 and P.size > 0)
    pins[k][0] ^= 1
    items = [(pw, d, x, x.numel(), y, w.size) for (pw, d, _), x, y, w in zip(msgs, pins, pouts, want)]
    st = np.full(len(items), -1, dtype=np.int32)
    lc.check(lc.lc_run_batch_host(ctx.handle, lc.Batch(items), st))
    for i, (y, w) in enumerate(zip(pouts, want)):
        if i == k:
            assert st[i] == lc.LC_ERR_INTEGRITY and not y.numpy().any()
        else:
            assert st[i] == 0 and np.array_equal(y.numpy()[:w.size], w), i


def _host_batch(seed, count, pinned=True, tamper=False):
    """(Batch, status array, output buffers, expected outputs, refs)."""
    msgs = _mixed_batch(count, seed, max_size=3 * B + 100)
    ins, want = [], []
    for pw, d, P in msgs:
        ct = O.encrypt(pw, P)
        ins.append(P if d == 0 else ct.copy())
        want.append(ct if d == 0 else P)
    bad = None
    if tamper:
        bad = next(i for i, (_, d, P) in enumerate(msgs) if d == 1 and P.size > 0)
        ins[bad][0] ^= 1
    if pinned:
        hin = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in ins]
        hout = [torch.full((max(1, w.size),), 0xAA, dtype=torch.uint8).pin_memory() for w in want]
        items = [(pw, d, x, x.numel(), y, w.size) for (pw, d, _), x, y, w in zip(msgs, hin, hout, want)]
        outs = [y.numpy() for y in hout]
    else:
        hin = [np.ascontiguousarray(x) for x in ins]
        outs = [np.full(max(1, w.size), 0xAA, dtype=np.uint8) for w in want]
        items = [(pw, d, x, x.size, y, w.size) for (pw, d, _), x, y, w in zip(msgs, hin, outs, want)]
    st = np.full(len(items), -1, dtype=np.int32)
    return lc.Batch(items), st, outs, want, bad, (hin, outs)


def _check_host_batch(st, outs, want, bad):
    for i, (y, w) in enumerate(zip(outs, want)):
        if i == bad:
            assert st[i] == lc.LC_ERR_INTEGRITY and not y[:w.size].any(), i
        else:
            assert st[i] == lc.LC_OK and np.array_equal(y[:w.size], w), i


def test_submitted_host_batches_overlap_and_match_oracle(ctx):
    h = ctx.handle
    assert lc.lc_wait_batch_host(h, 0) == lc.LC_ERR_ARG
    batches = [_host_batch(900 + k, 12 + 3 * k, pinned=(k != 3), tamper=(k == 1)) for k in range(6)]
    tickets = []
    for k, (bt, st, outs, want, bad, refs) in enumerate(batches):
        rc, t = lc.lc_submit_batch_host(h, bt, st)
        assert rc == lc.LC_OK and t > 0
        tickets.append(t)
        if k == 2:
            # a synchronous host batch and a device batch between submissions
            sb, sst, souts, swant, sbad, _ = _host_batch(950, 9)
            lc.check(lc.lc_run_batch_host(h, sb, sst))
            _check_host_batch(sst, souts, swant, sbad)
            gpu_out = gpu_encrypt(ctx, b"between", synth.uniform_bytes(951, 5 * B + 3))
            assert np.array_equal(gpu_out, O.encrypt(b"between", synth.uniform_bytes(951, 5 * B + 3)))
    assert tickets == sorted(tickets) and len(set(tickets)) == len(tickets)
    assert lc.lc_wait_batch_host(h, tickets[-1] + 1) == lc.LC_ERR_ARG
    # waiting for the fifth ticket completes every earlier batch too
    assert lc.lc_wait_batch_host(h, tickets[4]) == lc.LC_OK
    for k in range(5):
        _, st, outs, want, bad, _ = batches[k]
        _check_host_batch(st, outs, want, bad)
    assert lc.lc_wait_batch_host(h, tickets[5]) == lc.LC_OK
    _, st, outs, want, bad, _ = batches[5]
    _check_host_batch(st, outs, want, bad)
    # waiting again is a no-op; an empty batch gets a completed ticket
    assert lc.lc_wait_batch_host(h, tickets[2]) == lc.LC_OK
    rc, t = lc.lc_submit_batch_host(h, lc.Batch([]), np.zeros(1, np.int32))
    assert rc == lc.LC_OK and t > tickets[-1]
    assert lc.lc_wait_batch_host(h, t) == lc.LC_OK


def test_chunked_host_batch(ctx):
    # A host-buffer batch larger than host_chunk_mib is cut into up to 4
    # chunks whose copies overlap the other chunks' kernels; results are
    # those of the oracle, in one synchronous call and in pipelined submits.
    rng = np.random.default_rng(71)
    msgs = []
    for m in range(48):
        n = int(rng.integers(1, 200 * 1024))
        pw = synth.password(synth.subseed(72, m), 8 + m % 25)
        P = synth.uniform_bytes(synth.subseed(73, m), n)
        msgs.append((pw, m % 2, P))
    ins, want = [], []
    for pw, d, P in msgs:
        ct = O.encrypt(pw, P)
        ins.append(P if d == 0 else ct)
        want.append(ct if d == 0 else P)
    assert sum(x.size for x in ins) > 4 << 20
    hin = torch.empty(sum(x.size for x in ins), dtype=torch.uint8).pin_memory()
    a = 0
    offs = []
    for x in ins:
        hin[a:a + x.size] = torch.from_numpy(x)
        offs.append(a)
        a += x.size
    try:
        assert lc.lc_ctx_set_launch(ctx.handle, 256, 0, 0, 0, 1) == lc.LC_OK
        for rep in range(3):
            hout = torch.full((sum(w.size for w in want),), 0x33, dtype=torch.uint8).pin_memory()
            items, b_ = [], 0
            for (pw, d, _), x, o, w in zip(msgs, ins, offs, want):
                items.append((pw, d, hin.data_ptr() + o, x.size, hout.data_ptr() + b_, w.size))
                b_ += w.size
            st = np.full(len(items), -1, dtype=np.int32)
            if rep == 0:
                lc.check(lc.lc_run_batch_host(ctx.handle, lc.Batch(items), st))
            else:
                rc, t = lc.lc_submit_batch_host(ctx.handle, lc.Batch(items), st)
                assert rc == lc.LC_OK
                assert lc.lc_wait_batch_host(ctx.handle, t) == lc.LC_OK
            assert (st == 0).all(), rep
            got = hout.numpy()
            b_ = 0
            for w in want:
                assert np.array_equal(got[b_:b_ + w.size], w), rep
                b_ += w.size
    finally:
        lc.lc_ctx_set_launch(ctx.handle, 256, 0)


def test_one_context_two_streams(ctx):
    # Batches of one context issued on two streams without host
    # synchronisation: each waits for the previous one on the GPU, because
    # they share the context's workspace.  Every result equals the oracle.
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    jobs = []
    for k in range(6):
        msgs = _mixed_batch(40, 300 + k, max_size=6 * B)
        ins, want = [], []
        for pw, d, P in msgs:
            ct = O.encrypt(pw, P)
            ins.append(dev(P if d == 0 else ct))
            want.append(ct if d == 0 else P)
        outs = [torch.full((max(1, w.size),), 0x77, dtype=torch.uint8, device="cuda") for w in want]
        items = [(pw, d, x, x.numel(), y, w.size) for (pw, d, _), x, y, w in zip(msgs, ins, outs, want)]
        st = torch.full((len(items),), -1, dtype=torch.int32, device="cuda")
        jobs.append((lc.Batch(items), st, ins, outs, want))
    torch.cuda.synchronize()
    for k, (b, st, _, _, _) in enumerate(jobs):
        strm = s1 if k % 2 == 0 else s2
        lc.check(lc.lc_run_batch(ctx.handle, b, st, lc.LC_PARALLEL, strm))
    torch.cuda.synchronize()
    for k, (_, st, _, outs, want) in enumerate(jobs):
        assert (host(st) == 0).all(), k
        for y, w in zip(outs, want):
            assert np.array_equal(host(y)[:w.size], w), k


def test_message_over_4gib(ctx):
    # One message just over 2^32 bytes: part offsets b * 4096 and tag offsets
    # n + 8 b pass 2^32.  Every byte of the last 16,384 parts (across the
    # boundary, up to the ragged last one) and of the first two parts equals
    # the oracle; the whole message round-trips.
    n = (1 << 32) + 3 * B + 5
    seed = 0x4_0000_0001
    pw = b"over-four-gibibytes"
    P = torch.empty(n, dtype=torch.uint8, device="cuda")
    lc.check(lc.lc_synth_uniform(P, n, seed, 0))
    Cd = ctx.encrypt(pw, P)
    nb = -(-n // B)
    assert Cd.numel() == n + T * nb
    key = O.key_schedule(pw)
    Ph = np.zeros(n, dtype=np.uint8)          # only the checked parts are filled
    Cb = np.zeros(n + T * nb, dtype=np.uint8)
    edge = (1 << 32) // B
    for b in (0, 1, nb - 2, nb - 1):
        lo, hi = b * B, min(n, (b + 1) * B)
        Ph[lo:hi] = synth.uniform_bytes(seed, hi - lo, lo)
        O.encrypt_blocks(key, Ph, n, Cb, b, b + 1)
        assert np.array_equal(host(Cd[lo:hi]), Cb[lo:hi]), b
        assert np.array_equal(host(Cd[n + T * b:n + T * b + T]), Cb[n + T * b:n + T * b + T]), b
    # every byte of the last 16,384 parts (the 64 MiB that end the message:
    # parts on both sides of the 2^32 boundary and the ragged last one) and
    # of their tags, the oracle on all cores
    b0, b1 = nb - 16384, nb
    assert b0 < edge < b1
    lo, hi = b0 * B, n
    Ph[lo:hi] = oracle_mt.uniform(seed, hi - lo, lo)
    jobs = [(c, min(b1, c + 64)) for c in range(b0, b1, 64)]
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(oracle_mt.THREADS) as ex:
        list(ex.map(lambda j: O.encrypt_blocks(key, Ph, n, Cb, j[0], j[1]), jobs))
    assert oracle_mt.first_difference(host(Cd[lo:hi]), Cb[lo:hi]) == -1
    assert oracle_mt.first_difference(host(Cd[n + T * b0:n + T * b1]), Cb[n + T * b0:n + T * b1]) == -1
    del Ph, Cb
    st, back = ctx.decrypt(pw, Cd)
    assert st == lc.LC_OK
    step = 1 << 30
    for a in range(0, n, step):
        assert torch.equal(back[a:a + step], P[a:a + step]), a


# ---------------------------------------------------------------------------
# per-request key material: lambda (Eq. 5) and k (Eq. 7)
# ---------------------------------------------------------------------------

KEYS = [
    (None, None),                                   # the context's (1, 1, 20), (4, 4, 4)
    ((-15.0, -11.0, 61.0), (3, 4, 3)),
    ((15.9, 15.9, 0.1), (3, 3, 3)),
    ((0.5, -2.25, 30.0), None),                     # lambda only: the v1 variant
    (None, (4, 3, 4)),
]


@pytest.mark.parametrize("mode", [lc.LC_PARALLEL, lc.LC_SEQUENTIAL])
@pytest.mark.parametrize("k_in_batch", [True, False], ids=["mixed-k", "lambda-only"])
@pytest.mark.parametrize("small", [0, 1], ids=["auto", "throughput-build"])
def test_per_request_lambda_and_k(ctx, mode, k_in_batch, small):
    # One batch mixes requests with their own (lambda, k) and with the
    # context's; each equals the oracle run with those parameters, in both
    # directions.  Without a k != 4 in the batch the v1 kernel variant runs;
    # with one, a small batch runs the general path and, with the small-batch
    # threshold at one part, the v1 build that reads k per message.
    try:
        assert lc.lc_ctx_set_launch(ctx.handle, 256, 0, 0, small) == lc.LC_OK
        _per_request_lambda_and_k(ctx, mode, k_in_batch)
    finally:
        lc.lc_ctx_set_launch(ctx.handle, 256, 0)


def _per_request_lambda_and_k(ctx, mode, k_in_batch):
    keys = KEYS if k_in_batch else [kk for kk in KEYS if kk[1] is None]
    items, expect, keep = [], [], []
    for i, n in enumerate([0, 1, 33, B, B + 1, 3 * B + 7, 20000, 70001]):
        for j, (lam, k) in enumerate(keys):
            pw = synth.password(synth.subseed(90, 10 * i + j), 4 + (3 * i + j) % 29)
            P = synth.uniform_bytes(synth.subseed(91, 10 * i + j), n)
            po = O.params(**({"lam": lam} if lam else {}), **({"k": k} if k else {}))
            ct = O.encrypt(pw, P, mode, po)
            d = (i + j) % 2
            src, want = (P, ct) if d == 0 else (ct, P)
            x = dev(src) if src.size else torch.zeros(1, dtype=torch.uint8, device="cuda")
            y = torch.full((max(1, want.size),), 0x3C, dtype=torch.uint8, device="cuda")
            keep += [x, y]
            items.append((pw, d, x if src.size else None, src.size, y, want.size, lam, k))
            expect.append(want)
    st = torch.full((len(items),), -1, dtype=torch.int32, device="cuda")
    lc.check(lc.lc_run_batch_ex(ctx.handle, lc.BatchEx(items), st, mode))
    assert (host(st) == 0).all()
    for it, want in zip(items, expect):
        assert np.array_equal(host(it[4])[:want.size], want), it[:2] + it[6:]
    # a wrong k is a wrong key: the decryption is rejected and zeroed
    pw, P = b"wrong-k", synth.uniform_bytes(92, 5000)
    ct = O.encrypt(pw, P, mode, O.params(k=(3, 3, 3)))
    x, y = dev(ct), torch.ones(P.size, dtype=torch.uint8, device="cuda")
    s1 = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    lc.check(lc.lc_run_batch_ex(ctx.handle, lc.BatchEx([(pw, 1, x, ct.size, y, P.size, None, (4, 3, 3))]),
                                s1, mode))
    assert host(s1)[0] == lc.LC_ERR_INTEGRITY and not host(y).any()


def test_pipe_probes_report_rates():
    # The microbenchmarks behind the roofline denominators and the
    # one-trajectory latency: positive rates; one DADD warp instruction per
    # warp issue interval whatever the number of active lanes.
    r = lc.lc_probe_pipes(0)
    assert r.sm_count > 0 and r.dadd_gops > 0 and r.ialu_gops > r.dadd_gops
    full = lc.lc_probe_fp64_warp(0, 1, 1, 32)
    one = lc.lc_probe_fp64_warp(0, 1, 1, 1)
    assert full > 4 and abs(full - one) / full < 0.1
    assert lc.lc_probe_fp64_warp(0, 8, 2, 32) > full  # eight warps share the SM's FP64 pipe
    with pytest.raises(lc.LcError):
        lc.lc_probe_fp64_warp(0, 33, 1, 32)
