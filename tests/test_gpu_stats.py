"""Ciphertext statistics (Sec. 4): the byte-statistics kernel against exact
numpy sums, and the paper's statistical claims on GPU ciphertexts."""
import numpy as np
import pytest

from paper_1201_3114_gb300 import lc, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = lc.Context(0)
    yield c
    c.close()


def _np_stats(x, max_lag):
    x = x.astype(np.uint64)
    hist = np.bincount(x.astype(np.int64), minlength=256)
    lag = [int((x[:-k] * x[k:]).sum()) if x.size > k else 0 for k in range(1, max_lag + 1)]
    return hist, int(x.sum()), int((x * x).sum()), lag


@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 100, 65536, 65536 * 3 + 7, 1 << 22])
def test_stats_exact(ctx, n):
    x = synth.zipf_text(60 + n % 97, n, zero_run=4096 if n > 8192 else 0)
    for shift in (0, 3):
        buf = torch.zeros(n + 16, dtype=torch.uint8, device="cuda")
        if n:
            buf[shift:shift + n] = torch.from_numpy(x).cuda()
        for max_lag in (0, 1, 8):
            st = lc.lc_byte_stats(ctx.handle, buf.data_ptr() + shift, n, max_lag)
            hist, s1, s2, lag = _np_stats(x, max_lag)
            assert st.n == n
            assert list(st.hist) == list(hist)
            assert (st.sum, st.sum_sq) == (s1, s2)
            assert list(st.lag_sum)[:max_lag] == lag


def _periodic_stats(n, period, max_lag):
    """Exact statistics of x_i = i mod period, i = 0..n-1, in closed form:
    whole periods times the sums over one period, plus the partial one."""
    q, r = divmod(n, period)
    hist = [q + (1 if v < r else 0) if v < period else 0 for v in range(256)]
    lag = []
    for k in range(1, max_lag + 1):
        m = max(n - k, 0)
        qk, rk = divmod(m, period)
        one = sum(j * ((j + k) % period) for j in range(period))
        lag.append(qk * one + sum(j * ((j + k) % period) for j in range(rk)))
    return hist, lag


@pytest.mark.parametrize("shift", [0, 3])
def test_stats_closed_form_6gib(ctx, shift):
    # 6 GiB: every thread of both builds walks hundreds of grid strides, and
    # the lagged build's 32-bit partials go through their periodic flush into
    # the 64-bit totals (every 1024 chunks per thread)
    n, period = 6 << 30, 251
    buf = torch.empty(n + 16, dtype=torch.uint8, device="cuda")
    pat = torch.arange(period, device="cuda").to(torch.uint8)
    reps = (n + period - 1) // period
    buf[shift:shift + n] = pat.repeat(reps)[:n]
    for max_lag in (0, 8):
        st = lc.lc_byte_stats(ctx.handle, buf.data_ptr() + shift, n, max_lag)
        hist, lag = _periodic_stats(n, period, max_lag)
        assert st.n == n
        assert list(st.hist) == hist
        assert st.sum == sum(v * c for v, c in enumerate(hist))
        assert list(st.lag_sum)[:max_lag] == lag
    del buf
    torch.cuda.empty_cache()


def test_ciphertext_statistics(ctx):
    # Sec. 4: the ciphertext histogram is flat and carries no correlation
    # between neighbouring bytes; two close passwords give unrelated
    # ciphertexts.  Under the Step-3 reading every part reaches the absorbing
    # (mu, Omega) lock, after which C - P = 2 R is even: the ciphertext's low
    # bit is the plaintext's.  So for text the entropy is bounded by
    # 7 + H(low bit of P) (the 7/16 bias of R mod 4 keeps it slightly below),
    # and for uniform data it is 8.
    n = 1 << 22
    P = torch.from_numpy(synth.zipf_text(61, n)).cuda()
    ps = lc.lc_byte_stats(ctx.handle, P, n)
    c1 = ctx.encrypt(b"123456", P)
    c2 = ctx.encrypt(b"123457", P)
    cs = lc.lc_byte_stats(ctx.handle, c1, n)
    h = np.array(ps.hist, dtype=np.float64)
    p1 = h[1::2].sum() / n
    h_lsb = -(p1 * np.log2(p1) + (1 - p1) * np.log2(1 - p1))
    assert lc.entropy_bits(ps) < 5.5
    Hc = lc.entropy_bits(cs)
    assert 7.95 < Hc <= 7 + h_lsb + 1e-3, (Hc, h_lsb)
    assert all(abs(r) < 0.01 for r in lc.autocorrelation(cs))
    assert (c1[:n] != c2[:n]).float().mean().item() > 0.99
    U = torch.empty(n, dtype=torch.uint8, device="cuda")
    lc.check(lc.lc_synth_uniform(U, n, 62, 0))
    cu = lc.lc_byte_stats(ctx.handle, ctx.encrypt(b"uniform", U), n)
    assert lc.entropy_bits(cu) > 7.999


# ---------------------------------------------------------------------------
# Fig. 1: digit statistics of the trajectory coordinates
# ---------------------------------------------------------------------------

def _oracle_digits(msgs, prm):
    """The oracle's Fig. 1 counts over the encryption of (pw, P) messages in
    parallel mode."""
    import oracle as O
    st = O.Stats()
    for pw, P in msgs:
        key = O.key_schedule(pw, prm)
        n = P.size
        Cb = np.zeros(O.ciphertext_len(n, prm=prm), np.uint8)
        O.encrypt_blocks(key, np.ascontiguousarray(P), n, Cb, 0, O.nblocks(n, prm=prm), prm, st)
    return st.digit_arrays(), int(st.steps)


@pytest.mark.parametrize("over", [{}, {"dt": 0.027}, {"k": (3, 4, 4), "steps_per_byte": 2}],
                         ids=["v1", "dt0.027", "general"])
def test_fig1_digit_stats_match_oracle(over):
    # Every count of the counting kernels equals the oracle's over the same
    # encryptions; decrypting the ciphertexts follows the same trajectories,
    # so it doubles every count.  The outputs are unchanged by counting.
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
    prm = O.params(**over)
    sizes = [1, 100, 4096, 4097, 3 * 4096 + 77, 70000]
    msgs = [(synth.password(synth.subseed(80, i), 5 + i), synth.uniform_bytes(synth.subseed(81, i), n))
            for i, n in enumerate(sizes)]
    (want_ip, want_dg, want_oor), steps = _oracle_digits(msgs, prm)
    with lc.Context(0, lc.params(**over)) as c:
        ins = [torch.from_numpy(P).cuda() for _, P in msgs]
        outs = [torch.zeros(c.ciphertext_len(P.size), dtype=torch.uint8, device="cuda") for _, P in msgs]
        items = [(pw, 0, x, x.numel(), y, y.numel()) for (pw, _), x, y in zip(msgs, ins, outs)]
        st = torch.full((len(items),), -1, dtype=torch.int32, device="cuda")
        lc.check(lc.lc_ctx_digit_stats(c.handle, True))
        lc.check(lc.lc_run_batch(c.handle, lc.Batch(items), st))
        d = lc.lc_ctx_get_digit_stats(c.handle)
        assert (st.cpu().numpy() == 0).all()
        ip, dg, oor = d.arrays()
        assert d.states == steps
        assert np.array_equal(ip, want_ip) and np.array_equal(dg, want_dg)
        assert np.array_equal(oor, want_oor)
        for (pw, P), y in zip(msgs, outs):
            assert np.array_equal(y.cpu().numpy(), O.encrypt(pw, P, O.PARALLEL, prm))
        # decrypting (still counting) adds the same counts again
        backs = [torch.zeros(max(1, P.size), dtype=torch.uint8, device="cuda") for _, P in msgs]
        items = [(pw, 1, y, y.numel(), b, P.size) for (pw, P), y, b in zip(msgs, outs, backs)]
        lc.check(lc.lc_run_batch(c.handle, lc.Batch(items), st))
        ip2, dg2, oor2 = lc.lc_ctx_get_digit_stats(c.handle).arrays()
        assert (st.cpu().numpy() == 0).all()
        assert np.array_equal(ip2, 2 * want_ip) and np.array_equal(dg2, 2 * want_dg)
        assert np.array_equal(oor2, 2 * want_oor)
        # counting off: the counters stay, the kernels go back to the fast build
        lc.check(lc.lc_ctx_digit_stats(c.handle, False))
        lc.check(lc.lc_run_batch(c.handle, lc.Batch(items), st))
        assert np.array_equal(lc.lc_ctx_get_digit_stats(c.handle).arrays()[0], 2 * want_ip)
        if over.get("dt") == 0.027:
            assert int(want_oor.sum()) > 0  # the divergent profile reaches |v| >= 2^31


# ---------------------------------------------------------------------------
# Sec. 4 statistics fused into the cipher kernel
# ---------------------------------------------------------------------------

def _sum_np_stats(cts):
    """Sum over ciphertexts of their exact byte statistics (pairs inside one
    ciphertext only)."""
    hist = np.zeros(256, dtype=np.int64)
    s1 = s2 = n = 0
    lag = [0] * 8
    for c in cts:
        h, a, b, l8 = _np_stats(c, 8)
        hist += h
        s1, s2, n = s1 + a, s2 + b, n + c.size
        lag = [x + y for x, y in zip(lag, l8)]
    return n, hist, s1, s2, lag


@pytest.mark.parametrize("mode", [lc.LC_PARALLEL, lc.LC_SEQUENTIAL], ids=["parallel", "sequential"])
@pytest.mark.parametrize("over", [{}, {"k": (3, 4, 4)}, {"block_len": 16, "tag_len": 3}],
                         ids=["v1", "general", "short-segments"])
def test_fused_ciphertext_stats(mode, over):
    # The counting build's statistics equal the exact statistics of the
    # oracle's ciphertexts (encryptions only; the decryptions in the same
    # batch add nothing), and its outputs equal the oracle's.  Sizes cover
    # empty and one-byte messages, a last part shorter than the lag window,
    # whole parts and ragged tails; the inputs sit at odd offsets so that
    # the single-byte head path counts too.  block_len = 16 with 3-byte tags
    # makes most segments shorter than 8 bytes, so pairs span several
    # segment starts.
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
    prm = O.params(**over)
    B = prm.block_len
    sizes = [0, 1, 5, B - 1, B, B + 3, 3 * B + 5, 4096 * 3 + 17, 70001, 262144 + 9]
    msgs = [(synth.password(synth.subseed(90, i), 4 + (5 * i) % 29), synth.uniform_bytes(synth.subseed(91, i), n))
            for i, n in enumerate(sizes)]
    want_c = [O.encrypt(pw, P, mode, prm) for pw, P in msgs]
    with lc.Context(0, lc.params(**over)) as c:
        items, outs, keep = [], [], []
        for i, ((pw, P), ct) in enumerate(zip(msgs, want_c)):
            off = 1 + i % 7
            src = torch.zeros(P.size + off, dtype=torch.uint8, device="cuda")
            if P.size:
                src[off:] = torch.from_numpy(P).cuda()
            dst = torch.full((ct.size,), 0xEE, dtype=torch.uint8, device="cuda")
            keep.append(src)
            items.append((pw, lc.LC_ENCRYPT, src.data_ptr() + off, P.size, dst, dst.numel()))
            outs.append(dst)
            # a decryption of the oracle's ciphertext in the same batch
            cin = torch.from_numpy(ct).cuda()
            back = torch.zeros(max(1, P.size), dtype=torch.uint8, device="cuda")
            keep += [cin, back]
            items.append((pw, lc.LC_DECRYPT, cin, cin.numel(), back, P.size))
        st = torch.full((len(items),), -1, dtype=torch.int32, device="cuda")
        lc.check(lc.lc_ctx_ciphertext_stats(c.handle, True))
        for rep in (1, 2):
            lc.check(lc.lc_run_batch(c.handle, lc.Batch(items), st, mode))
            got = lc.lc_ctx_get_ciphertext_stats(c.handle)
            assert (st.cpu().numpy() == 0).all()
            for y, ct in zip(outs, want_c):
                assert np.array_equal(y.cpu().numpy(), ct)
            n, hist, s1, s2, lag = _sum_np_stats(want_c)
            assert got.n == rep * n
            assert list(got.hist) == list(rep * hist)
            assert (got.sum, got.sum_sq) == (rep * s1, rep * s2)
            assert list(got.lag_sum) == [rep * x for x in lag]
        # one message through lc_encrypt equals the separate pass over its
        # ciphertext; counting off leaves the totals alone
        lc.check(lc.lc_ctx_ciphertext_stats(c.handle, True))
        pw, P = msgs[-1]
        C1 = c.encrypt(pw, torch.from_numpy(P).cuda(), mode)
        fused = lc.lc_ctx_get_ciphertext_stats(c.handle)
        sep = lc.lc_byte_stats(c.handle, C1, C1.numel())
        assert (fused.n, list(fused.hist), list(fused.lag_sum)) == (sep.n, list(sep.hist), list(sep.lag_sum))
        lc.check(lc.lc_ctx_ciphertext_stats(c.handle, False))
        c.encrypt(pw, torch.from_numpy(P).cuda(), mode)
        assert lc.lc_ctx_get_ciphertext_stats(c.handle).n == sep.n
