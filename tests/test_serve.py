"""Serving loop: the arena's admission accounting and the serving policy on
a simulated device (CPU), and a small served workload on the GPU (verdicts,
plaintexts, alone-vs-mix equality)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1201_3114_gb300 import lc, serve, synth  # noqa: E402


def test_arena_buddy_split_merge_and_budget():
    a = serve.Arena(128 << 20, "cpu")            # two 64 MiB top blocks
    assert a.cap == 128 << 20
    b1 = a.alloc(5000)                            # 8 KiB block
    b2 = a.alloc(100)                             # 4 KiB block (minimum)
    assert a.in_use == 8192 + 4096
    big = [a.alloc(64 << 20) for _ in range(2)]
    assert big[0] is not None and big[1] is None  # one top block is split
    a.release(big[0])
    a.release(b1)
    a.release(b2)
    assert a.in_use == 0
    # everything merged back: both top blocks are whole again
    assert len(a.free[a.MAX_CLASS]) == 2
    assert all(not a.free[k] for k in range(a.MIN_CLASS, a.MAX_CLASS))
    # fill with minimum blocks: exactly cap / 4 KiB fit, then admission waits
    blocks = [a.alloc(4096) for _ in range((128 << 20) // 4096)]
    assert all(b is not None for b in blocks) and a.alloc(1) is None
    assert len({b[0] for b in blocks}) == len(blocks)
    for b in blocks[::2]:
        a.release(b)
    assert a.alloc(8192) is None                  # free space is fragmented
    for b in blocks[1::2]:
        a.release(b)
    assert a.alloc(64 << 20) is not None and a.in_use == 64 << 20
    with pytest.raises(ValueError):
        a.alloc((64 << 20) + 1)


class _FakeArena(serve.Arena):
    """Host arena that forgets a block's tampered mark when it is released."""

    def __init__(self, nbytes, tampered):
        super().__init__(nbytes, "cpu")
        self.tampered = tampered

    def release(self, blk):
        self.tampered.discard(blk[0])
        super().release(blk)


class FakeBackend:
    """CPU stand-in for serve.CudaBackend, for testing the serving policy
    without a GPU.  It does no cipher arithmetic: batches share one device
    that works through their bytes at a fixed rate, each with a fixed
    latency on top; encryptions succeed, and a
    decryption fails its verdict exactly when its input block was made by
    tamper_copy.  Each launch checks the policy's invariants."""

    def __init__(self, streams=3, budget_bytes=128 << 20, pool_bytes=1 << 20, gbps=2.0,
                 latency_ms=1.0):
        self.tampered = set()
        self.arena = _FakeArena(budget_bytes, self.tampered)
        self.pool_bytes = pool_bytes
        self.pool_base = 1 << 44  # an address that is never dereferenced
        self.nstreams = streams
        self.rate = gbps * 1e9
        self.latency = latency_ms * 1e-3
        self.running = [None] * streams
        self.verified = 0
        self.device_free = 0.0
        self.status = [None] * streams
        self.launches = 0
        self.batches = []  # (slot, requests, input bytes, start, finish)

    def start(self):
        self.t0 = time.perf_counter()
        self.device_free = 0.0

    def clock(self):
        return time.perf_counter() - self.t0

    def launch(self, s, reqs, count):
        assert self.running[s] is None or self.done(self.running[s]), "slot busy"
        r = reqs[:count]
        outs = set()
        for k in range(count):
            off = int(r["out"][k]) - self.arena.base
            assert 0 <= off and off + int(r["out_cap"][k]) <= self.arena.cap, "output outside the arena"
            assert off not in outs, "two requests share an output block"
            outs.add(off)
            src = int(r["inp"][k])
            if r["dir"][k] == 0:
                assert self.pool_base <= src and src + int(r["in_len"][k]) <= self.pool_base + self.pool_bytes
            else:
                assert 0 <= src - self.arena.base < self.arena.cap, "decrypt input outside the arena"
        nbytes = int(r["in_len"].sum())
        now = self.clock()
        # one device shared by all slots: batches take turns at the byte
        # rate, each with a fixed latency on top
        begin = max(now, self.device_free)
        self.device_free = begin + nbytes / self.rate
        token = {"finish": self.device_free + self.latency}
        st = np.zeros(count, dtype=np.int32)
        for k in range(count):
            if r["dir"][k] == 1 and int(r["inp"][k]) - self.arena.base in self.tampered:
                st[k] = lc.LC_ERR_INTEGRITY
        self.running[s] = token
        self.status[s] = st
        self.launches += 2
        self.batches.append((s, count, nbytes, now, token["finish"]))
        return token

    def done(self, token):
        return self.clock() >= token["finish"]

    def finish_ms(self, token):
        return token["finish"] * 1e3

    def statuses(self, s, count):
        return self.status[s][:count].copy()

    def tamper_copy(self, s, dst, src, nbytes, pos):
        assert dst != src and 0 <= pos < nbytes
        self.tampered.add(dst[0])

    def read(self, blk, n):
        return np.zeros(n, dtype=np.uint8)

    def capture_reserve(self, nbytes):
        self.cap_left = nbytes

    def capture_async(self, s, blk, n):
        assert 0 <= blk[0] and blk[0] + n <= self.arena.cap and n <= self.cap_left
        self.cap_left -= n
        return np.zeros(n, dtype=np.uint8)

    def equals_pool(self, blk, n, off):
        return True

    def verify_async(self, s, blk, n, off):
        assert 0 <= blk[0] and blk[0] + n <= self.arena.cap and 0 <= off and off + n <= self.pool_bytes
        self.verified += 1

    def fence(self, s):
        # done once slot s's latest batch has finished
        run = self.running[s]
        return {"finish": run["finish"] if run is not None else 0.0}

    def mismatches(self):
        return 0

    def sync(self):
        pass

    def launch_count(self):
        return self.launches

    def close(self):
        pass


def _serve_fake(spec, **kw):
    be_kw = {k: kw.pop(k) for k in ("budget_bytes", "gbps", "latency_ms", "streams", "pool_bytes")
             if k in kw}
    be = FakeBackend(**be_kw)
    srv = serve.Server(backend=be, **kw)
    w = serve.Workload(spec)
    return w, be, srv.run(w, poll=0.0001)


def test_serving_policy_on_fake_backend():
    # Admission, batching and the replay ring on a simulated device: every
    # request completes with the right verdict, no arena block leaks, batches
    # respect the byte cap, and batches on different slots overlap in time.
    spec = synth.cfg5_spec(rate=3000.0, duration=1.0, lo=256, hi=1 << 20, tamper_frac=0.05)
    w, be, st = _serve_fake(spec, budget_bytes=256 << 20, gbps=4.0, latency_ms=2.0,
                            max_batch_bytes=8 << 20, max_batch_requests=512)
    assert st["completed"] == w.n > 2000
    assert st["tampered"] > 0 and st["tampered_rejected"] == st["tampered"]
    assert st["untampered_decrypts_ok"] == st["untampered_decrypts"] > 0
    assert st["encrypts_ok"] == int((w.kind == 0).sum())
    assert be.arena.in_use == 0 and not be.tampered       # everything released
    assert st["arena_peak_bytes"] <= be.arena.cap
    assert st["max_batch_bytes"] <= 4 * (8 << 20) + (1 << 20)  # adaptive cap plus one request
    lat = st["done_ms"] - 1e3 * w.t
    assert (lat >= 2.0 - 1e-6).all()                      # no request beats the device
    assert st["p99_ms"] >= st["p50_ms"] >= 2.0
    overlap = sum(1 for a, b in zip(be.batches, be.batches[1:]) if b[3] < a[4] and b[0] != a[0])
    assert overlap > 0


def test_serving_backpressure_small_budget():
    # A 64 MiB budget against requests up to 16 MiB arriving faster than the
    # simulated device serves them: admission waits for memory, the queue
    # drains, and the budget is never exceeded.
    spec = synth.cfg5_spec(rate=400.0, duration=0.5, lo=1 << 20, hi=16 << 20, tamper_frac=0.1)
    w, be, st = _serve_fake(spec, budget_bytes=64 << 20, gbps=1.0, latency_ms=1.0,
                            max_batch_bytes=32 << 20, max_batch_requests=64, pool_bytes=32 << 20)
    assert st["completed"] == w.n
    assert st["arena_peak_bytes"] <= 64 << 20
    assert be.arena.in_use == 0
    assert st["tampered_rejected"] == st["tampered"]
    # ~2.2 GB/s offered against a 1 GB/s device: the queue grows and drains
    assert st["p99_ms"] > 100.0 and st["wall_s"] > 0.8


def test_small_first_policy_on_fake_backend():
    # Over capacity (about 1.2x a simulated 0.9 GB/s device) a backlog builds.
    # Serving the smallest size class first keeps small requests out of it,
    # so the median latency falls well below that of arrival order; every
    # verdict stays right, and decryptions replay ciphertexts of their own
    # size class.
    spec = synth.cfg5_spec(rate=2500.0, duration=1.0, lo=256, hi=4 << 20, tamper_frac=0.05)
    res = {}
    for policy in ("fifo", "small_first"):
        w, be, st = _serve_fake(spec, budget_bytes=512 << 20, gbps=0.9, latency_ms=2.0,
                                max_batch_bytes=8 << 20, max_batch_requests=1024,
                                pool_bytes=8 << 20, policy=policy, max_adaptive_bytes=0)
        assert st["completed"] == w.n and be.arena.in_use == 0
        assert st["tampered_rejected"] == st["tampered"] > 0
        assert st["untampered_decrypts_ok"] == st["untampered_decrypts"]
        dec = np.flatnonzero(w.kind == 1)
        same = np.array([serve.size_class(st["n_plain"][i]) == serve.size_class(w.size[i])
                         for i in dec])
        assert same.mean() > 0.9
        res[policy] = st
    assert res["small_first"]["p50_ms"] < 0.6 * res["fifo"]["p50_ms"]


def test_adaptive_cap_grows_batches_only_under_a_backlog():
    spec = synth.cfg5_spec(rate=2500.0, duration=0.6, lo=256, hi=4 << 20, tamper_frac=0.05)
    # over capacity: a backlog builds and batches grow past the 8 MiB cap
    w, be, st = _serve_fake(spec, budget_bytes=512 << 20, gbps=0.8, latency_ms=2.0,
                            max_batch_bytes=8 << 20, pool_bytes=8 << 20)
    assert st["completed"] == w.n and be.arena.in_use == 0
    assert (8 << 20) + (4 << 20) < st["max_batch_bytes"] <= (32 << 20) + (4 << 20)
    # well under capacity: no backlog, batches stay at the cap
    w, be, st = _serve_fake(spec, budget_bytes=512 << 20, gbps=20.0, latency_ms=2.0,
                            max_batch_bytes=8 << 20, pool_bytes=8 << 20)
    assert st["completed"] == w.n
    assert st["max_batch_bytes"] <= (8 << 20) + (4 << 20)


def test_serving_rejects_requests_larger_than_the_pool():
    spec = synth.cfg5_spec(rate=200.0, duration=0.2, lo=2 << 20, hi=4 << 20, tamper_frac=0.0)
    with pytest.raises(ValueError):
        _serve_fake(spec, pool_bytes=1 << 20)


def _small_spec(rate=2000.0, duration=1.5, lo=256, hi=16 << 20, tamper=0.05):
    s = synth.cfg5_spec(rate=rate, duration=duration, lo=lo, hi=hi, tamper_frac=tamper)
    return s


def test_capture_sample_spans_size_classes():
    w = serve.Workload(synth.cfg5_spec(rate=20000.0, duration=2.0))
    pick = serve.capture_sample(w, 8)
    assert pick == sorted(set(pick)) and all(w.kind[i] == 0 for i in pick)
    cls = {serve.size_class(int(w.size[i])) for i in pick}
    # 256 B - 16 MiB: class 0 (<= 256 B) and the classes (2^(7+c), 2^(8+c)], c = 1..16
    assert cls == set(range(0, 17)), sorted(cls)
    assert serve.capture_sample(w, 8) == pick  # seeded


def test_capture_on_fake_backend_holds_blocks():
    spec = synth.cfg5_spec(rate=800.0, duration=0.5, lo=256, hi=1 << 20, tamper_frac=0.05)
    be = FakeBackend(budget_bytes=256 << 20, pool_bytes=2 << 20, gbps=5.0)
    srv = serve.Server(backend=be)
    w = serve.Workload(spec)
    pick = serve.capture_sample(w, 4)
    st = srv.run(w, capture=pick, poll=0.0001)
    assert st["completed"] == w.n and set(st["captured"]) == set(pick)
    assert be.arena.in_use == 0 and be.cap_left == 0


@pytest.mark.gpu
def test_served_workload_verdicts_oracle_and_alone_vs_mix():
    # Sizes 256 B - 16 MiB as in the served configuration.  All verdicts,
    # every decrypted plaintext, and a sample of encryptions spread over every
    # size class: byte for byte against the oracle (plaintexts regenerated on
    # the host from the pool's seed) and against the same request run alone.
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle_mt
    w = serve.Workload(_small_spec())
    capture = serve.capture_sample(w, 8)
    srv = serve.Server(0, streams=6, budget_bytes=4 << 30, pool_bytes=64 << 20,
                       max_batch_bytes=64 << 20, max_batch_requests=1024)
    try:
        st = srv.run(w, capture=capture, verify_every=1)
        assert st["completed"] == w.n
        assert st["tampered"] > 0 and st["tampered_rejected"] == st["tampered"]
        assert st["untampered_decrypts_ok"] == st["untampered_decrypts"] > 0
        assert st["encrypts_ok"] == int((w.kind == 0).sum())
        assert st["plaintext_mismatches"] == 0 and st["plaintext_checked"] > 100
        assert st["batches"] > 3 and st["p99_ms"] >= st["p50_ms"] > 0
        assert len(capture) >= 100 and max(w.size[capture]) > (8 << 20)
        msgs, offs = [], []
        for i in capture:
            n = int(w.size[i])
            off = srv.plain_offset(w, i, n)
            offs.append(off)
            msgs.append((w.pw(i), synth.uniform_bytes(srv.be.pool_seed, n, off)))
        want = oracle_mt.encrypt_many(msgs)
        with lc.Context(0) as ctx:
            for k, i in enumerate(capture):
                n = int(w.size[i])
                assert np.array_equal(st["captured"][i], want[k]), (i, n)
                alone = ctx.encrypt(w.pw(i), srv.be.pool[offs[k]:offs[k] + n]).cpu().numpy()
                assert np.array_equal(alone, want[k]), (i, n)
    finally:
        srv.close()
