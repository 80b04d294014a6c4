"""Serving loop: the arena's admission accounting (CPU) and a small served
workload on the GPU (verdicts, plaintexts, alone-vs-mix equality)."""
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


def _small_spec(rate=2000.0, duration=1.5, lo=256, hi=256 << 10, tamper=0.05):
    s = synth.cfg5_spec(rate=rate, duration=duration, lo=lo, hi=hi, tamper_frac=tamper)
    return s


@pytest.mark.gpu
def test_served_workload_verdicts_and_alone_vs_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
    w = serve.Workload(_small_spec())
    enc = np.flatnonzero(w.kind == 0)
    capture = set(int(i) for i in enc[:: max(1, enc.size // 40)])
    srv = serve.Server(0, streams=3, budget_bytes=2 << 30, pool_bytes=64 << 20,
                       max_batch_bytes=32 << 20, max_batch_requests=1024)
    try:
        st = srv.run(w, capture=capture, verify_every=1)
        assert st["completed"] == w.n
        assert st["tampered"] > 0 and st["tampered_rejected"] == st["tampered"]
        assert st["untampered_decrypts_ok"] == st["untampered_decrypts"] > 0
        assert st["encrypts_ok"] == int((w.kind == 0).sum())
        assert st["plaintext_mismatches"] == 0 and st["plaintext_checked"] > 100
        assert st["batches"] > 3 and st["p99_ms"] >= st["p50_ms"] > 0
        # each captured encryption equals the same request run alone
        with lc.Context(0) as ctx:
            for i in sorted(capture):
                n = int(w.size[i])
                off = srv.plain_offset(w, i, n)
                alone = ctx.encrypt(w.pw(i), srv.pool[off:off + n]).cpu().numpy()
                assert np.array_equal(st["captured"][i], alone), i
                if n <= 16384:
                    P = srv.pool[off:off + n].cpu().numpy()
                    assert np.array_equal(alone, O.encrypt(w.pw(i), P)), i
    finally:
        srv.close()
