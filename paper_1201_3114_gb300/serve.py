"""Request serving with continuous batching over the batched cipher path.

Requests (encrypt or decrypt, any size, each with its own password) arrive
over time.  The loop admits them as device memory frees up, launches the
admitted ones as one lc_run_batch on a free stream, and records each
request's latency from arrival to GPU completion.  Every stream has its own
lc_ctx, so several batches are in flight at once.  When one batch's part
queue drains, its CTAs retire and the next batch's CTAs take the freed SMs:
requests that arrived while others were on the GPU overlap with them on the
device.  Admission is by a device-memory budget, an arena of that many bytes
carved into power-of-two blocks.  The batched path never changes the
arithmetic: a request gives the same bytes alone and in any mix.

Payloads live on the device: an encryption reads a slice of a
device-resident random pool, and a decryption replays the ciphertext of an
earlier completed encryption (a fraction with one byte flipped, which must
be rejected).  The host loop handles the bookkeeping only: all cipher work
runs in the library's kernels.
"""
import collections
import ctypes as C
import heapq
import math
import time

import numpy as np

from . import lc, synth

REQ_DTYPE = np.dtype([("pw", "<u8"), ("pw_len", "<u4"), ("dir", "<u4"), ("inp", "<u8"),
                      ("in_len", "<u8"), ("out", "<u8"), ("out_cap", "<u8")])
assert REQ_DTYPE.itemsize == C.sizeof(lc.lc_req)

B = 4096
T = 8


def ct_len(n):
    return n + T * max(1, -(-n // B))


NCLASS = 24  # size classes: [0, 256), [256, 512), ... by powers of two


def size_class(n):
    """Power-of-two size class of an n-byte message (0 for n <= 256)."""
    return min(NCLASS - 1, max(0, (max(1, int(n)) - 1).bit_length() - 8))


class Arena:
    """A device byte arena managed as a buddy system: blocks of 2^k bytes
    (4 KiB up to MAX_CLASS), split on allocation and merged with their free
    buddy on release, so no size mix strands memory.  Its size is the
    admission budget."""

    MIN_CLASS = 12
    MAX_CLASS = 26  # 64 MiB top blocks

    def __init__(self, nbytes, device):
        import torch
        top = 1 << self.MAX_CLASS
        nbytes = max(top, nbytes // top * top)
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)  # cpu in host tests
        self.base = self.buf.data_ptr()
        self.cap = nbytes
        self.free = {k: set() for k in range(self.MIN_CLASS, self.MAX_CLASS + 1)}
        self.free[self.MAX_CLASS] = set(range(0, nbytes, top))
        self.in_use = 0
        self.peak = 0

    def alloc(self, n):
        k = max(self.MIN_CLASS, (max(1, n) - 1).bit_length())
        if k > self.MAX_CLASS:
            raise ValueError("request of %d bytes exceeds the largest arena block" % n)
        j = k
        while j <= self.MAX_CLASS and not self.free[j]:
            j += 1
        if j > self.MAX_CLASS:
            return None
        off = self.free[j].pop()
        while j > k:  # split, keeping the lower half
            j -= 1
            self.free[j].add(off + (1 << j))
        self.in_use += 1 << k
        self.peak = max(self.peak, self.in_use)
        return off, k

    def release(self, blk):
        off, k = blk
        self.in_use -= 1 << k
        while k < self.MAX_CLASS:
            buddy = off ^ (1 << k)
            if buddy not in self.free[k]:
                break
            self.free[k].remove(buddy)
            off = min(off, buddy)
            k += 1
        self.free[k].add(off)

    def view(self, blk, n):
        return self.buf[blk[0]:blk[0] + n]


class Workload:
    """Served workload: arrival times, sizes, directions, tamper flags and
    passwords of every request (synth.cfg5_spec by default)."""

    def __init__(self, spec):
        self.t = np.asarray(spec["t"], dtype=np.float64)
        self.size = np.asarray(spec["sizes"], dtype=np.int64)
        self.kind = np.asarray(spec["kind"], dtype=np.int8)
        self.tamper = np.asarray(spec["tamper"], dtype=bool)
        self.data_seed = np.asarray(spec["data_seed"], dtype=np.uint64)
        self.flip_pos = np.asarray(spec["flip_pos"], dtype=np.uint64)
        self.pw_chars, self.pw_len = synth.passwords_bulk(spec["pw_seed"])
        self.pw_chars = np.ascontiguousarray(self.pw_chars)
        self.n = self.t.size

    def pw(self, i):
        return bytes(self.pw_chars[i, :self.pw_len[i]])


def capture_sample(w, per_class, seed=0xC0FFEE):
    """A seeded sample of encryption requests of ``w`` spread over every
    power-of-two size class: up to ``per_class`` per class, chosen by a
    seeded hash of the request index (for byte-level checks of served
    outputs)."""
    enc = np.flatnonzero(w.kind == 0)
    if enc.size == 0:
        return []
    order = np.argsort(synth.words(seed, 0, w.n)[enc], kind="stable")
    cls = np.array([size_class(n) for n in w.size[enc]])
    take, count = [], collections.Counter()
    for j in order:
        c = int(cls[j])
        if count[c] < per_class:
            count[c] += 1
            take.append(int(enc[j]))
    return sorted(take)


class CudaBackend:
    """The device side of the serving loop: one lc_ctx, CUDA stream and
    status buffer per stream slot, the device arena (admission budget) and
    the device-resident plaintext pool.  Every operation the loop needs from
    the device goes through these methods."""

    def __init__(self, device=0, streams=6, budget_bytes=48 << 30, pool_bytes=1 << 30,
                 max_batch_requests=8192, seed=0x5E4E, dense_build=1):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.ctxs = [lc.Context(device) for _ in range(streams)]
        # Batches on different streams share the GPU, so even a small batch
        # runs the throughput (integer-split) kernel variant, in its dense
        # build: 4 resident CTAs per SM let two right-sized batches (2 CTAs
        # per SM each) run side by side.
        for c in self.ctxs:
            lc.check(lc.lc_ctx_set_launch(c.handle, 256, 0, 0, 1, 0, dense_build), "lc_ctx_set_launch")
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.arena = Arena(budget_bytes, self.device)
        self.pool = torch.empty(pool_bytes, dtype=torch.uint8, device=self.device)
        self.pool_base = self.pool.data_ptr()
        self.pool_bytes = pool_bytes
        self.pool_seed = seed  # the pool is bytes [0, pool_bytes) of this uniform stream
        lc.check(lc.lc_synth_uniform(self.pool, pool_bytes, seed, 0, self.streams[0]))
        self.status_dev = [torch.zeros(max_batch_requests, dtype=torch.int32, device=self.device)
                           for _ in range(streams)]
        self.status_host = [torch.zeros(max_batch_requests, dtype=torch.int32).pin_memory()
                            for _ in range(streams)]
        torch.cuda.synchronize()
        self.warmup()

    @property
    def nstreams(self):
        return len(self.streams)

    def warmup(self, nbytes=32 << 20, seconds=1.0, busy_bytes=256 << 20):
        """Run one batch per stream before serving, so that graph capture and
        workspace growth do not land on the first requests; then keep every
        stream busy with full-size batches for `seconds`, so that serving
        starts on a GPU that has been under load."""
        torch = self.torch
        for k, n in enumerate((min(nbytes, self.pool_bytes), min(busy_bytes, self.pool_bytes))):
            outs = [torch.empty(ct_len(n), dtype=torch.uint8, device=self.device) for _ in self.ctxs]
            t0 = time.perf_counter()
            while True:
                for s, c in enumerate(self.ctxs):
                    lc.check(lc.lc_encrypt(c.handle, b"warm-up-password", self.pool_base, n,
                                           outs[s].data_ptr(), ct_len(n), lc.LC_PARALLEL,
                                           self.streams[s]), "warm-up")
                torch.cuda.synchronize()
                if k == 0 or time.perf_counter() - t0 >= seconds:
                    break
            del outs
        torch.cuda.empty_cache()

    def close(self):
        for c in self.ctxs:
            c.close()

    def start(self):
        """Mark time zero of a run (host clock and device clock)."""
        torch = self.torch
        self.base = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        self.base.record(self.streams[0])
        torch.cuda.synchronize()
        self.t0 = time.perf_counter()

    def clock(self):
        """Seconds since start()."""
        return time.perf_counter() - self.t0

    def launch(self, s, reqs, count):
        """Run requests reqs[:count] as one batch on stream slot s; returns a
        completion token."""
        torch = self.torch
        st = self.streams[s]
        ptr = reqs.ctypes.data_as(C.POINTER(lc.lc_req))
        rc = lc.load().lc_run_batch(self.ctxs[s].handle, ptr, count, self.status_dev[s].data_ptr(),
                                    lc.LC_PARALLEL, st.cuda_stream)
        lc.check(rc, "lc_run_batch")
        with torch.cuda.stream(st):
            self.status_host[s][:count].copy_(self.status_dev[s][:count], non_blocking=True)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(st)
        return ev

    def done(self, token):
        return token.query()

    def finish_ms(self, token):
        """Device time of the batch's completion, in ms since start()."""
        return self.base.elapsed_time(token)

    def statuses(self, s, count):
        return self.status_host[s].numpy()[:count].copy()

    def tamper_copy(self, s, dst, src, nbytes, pos):
        """dst <- src (arena blocks, nbytes), then flip byte pos, on slot s."""
        torch = self.torch
        v = self.arena.view(dst, nbytes)
        with torch.cuda.stream(self.streams[s]):
            v.copy_(self.arena.view(src, nbytes))
            v[pos:pos + 1].bitwise_xor_(0x5A)

    def read(self, blk, n):
        """Host copy of n bytes of an arena block (after its batch completed)."""
        return self.arena.view(blk, n).cpu().numpy()

    def capture_reserve(self, nbytes):
        """Page-locked host space for capture_async copies of one run."""
        self.cap_buf = self.torch.empty(max(1, nbytes), dtype=self.torch.uint8, pin_memory=True)
        self.cap_used = 0

    def capture_async(self, s, blk, n):
        """Copy n bytes of an arena block to the reserved host space on slot
        s's stream without waiting; returns the host array, valid after
        sync().  The block must not be reused before fence(s) is done."""
        a = self.cap_used
        if a + n > self.cap_buf.numel():
            raise ValueError("capture space exhausted")
        self.cap_used = a + n
        dst = self.cap_buf[a:a + n]
        with self.torch.cuda.stream(self.streams[s]):
            dst.copy_(self.arena.view(blk, n), non_blocking=True)
        return dst.numpy()

    def equals_pool(self, blk, n, off):
        """Whether n bytes of an arena block equal the pool at off (synchronous)."""
        return bool(self.torch.equal(self.arena.view(blk, n), self.pool[off:off + n]))

    def verify_async(self, s, blk, n, off):
        """Compare n bytes of an arena block with the pool at off on slot s's
        stream, counting a mismatch on the device; nothing waits.  The block
        must not be reused before fence(s)'s token is done."""
        torch = self.torch
        if not hasattr(self, "mismatch_dev"):
            self.mismatch_dev = torch.zeros(self.nstreams, dtype=torch.int32, device=self.device)
        with torch.cuda.stream(self.streams[s]):
            diff = torch.ne(self.arena.view(blk, n), self.pool[off:off + n]).any()
            self.mismatch_dev[s:s + 1].add_(diff.to(torch.int32).reshape(1))

    def fence(self, s):
        """A token that is done once the work enqueued on slot s so far is."""
        ev = self.torch.cuda.Event()
        ev.record(self.streams[s])
        return ev

    def mismatches(self):
        """Mismatches counted by verify_async (waits for the device)."""
        if not hasattr(self, "mismatch_dev"):
            return 0
        n = int(self.mismatch_dev.sum().item())
        self.mismatch_dev.zero_()
        return n

    def sync(self):
        self.torch.cuda.synchronize()

    def launch_count(self):
        return sum(lc.lc_ctx_launch_count(c.handle) for c in self.ctxs)


class Server:
    """Continuous-batching request loop over the backend's stream slots (a
    CudaBackend unless another backend is given)."""

    def __init__(self, device=0, streams=6, budget_bytes=48 << 30, pool_bytes=1 << 30,
                 max_batch_bytes=128 << 20, max_batch_requests=8192, replay_cap_bytes=None,
                 seed=0x5E4E, backend=None, policy="small_first", max_adaptive_bytes=None,
                 backlog_batches=4, dense_build=1):
        if policy not in ("fifo", "small_first"):
            raise ValueError("policy must be 'fifo' or 'small_first'")
        self.policy = policy
        self.be = backend if backend is not None else CudaBackend(
            device, streams, budget_bytes, pool_bytes, max_batch_requests, seed, dense_build)
        self.arena = self.be.arena
        self.max_batch_bytes = max_batch_bytes
        # Under a backlog (more than backlog_batches caps per slot waiting) a batch
        # may grow to a 1/slots share of the waiting bytes, up to this many
        # bytes (default 4x max_batch_bytes; 0 = off).  Bigger batches lose
        # less to their last partial wave, so the backlog drains instead of
        # settling into a slower regime.
        self.max_adaptive_bytes = (4 * max_batch_bytes if max_adaptive_bytes is None
                                   else max_adaptive_bytes)
        self.backlog_batches = backlog_batches
        self.max_batch_requests = max_batch_requests
        self.replay_cap = replay_cap_bytes if replay_cap_bytes is not None else self.arena.cap // 4
        self.reqs = [np.zeros(max_batch_requests, dtype=REQ_DTYPE) for _ in range(self.be.nstreams)]
        if backend is None:
            self.dry_run()

    def dry_run(self, seconds=3.0, rate=5000.0):
        """Serve a short synthetic workload at moderate load and discard the
        result.  The first run of the loop in a process was measured slow for
        its first seconds (every small device operation of the request path
        took ~10x longer on the host), and at a load near capacity the
        backlog it leaves does not drain; a second run in the same process
        was not affected."""
        spec = synth.cfg5_spec(rate=rate, duration=seconds, lo=256, hi=1 << 20, tamper_frac=0.02)
        self.run(Workload(spec), verify_every=8)

    def close(self):
        self.be.close()

    # ------------------------------------------------------------------
    def plain_offset(self, w, i, n):
        """Offset of request i's plaintext in the pool (16-byte aligned);
        n must not exceed the pool."""
        span = self.be.pool_bytes - n
        if span < 0:
            raise ValueError("request larger than the plaintext pool")
        return (int(w.data_seed[i]) % max(1, span)) & ~15 if span > 0 else 0

    def run(self, w: Workload, capture=(), verify_every=64, drain_timeout=60.0, poll=0.0002):
        """Serve every request of ``w``; returns a stats dict.  Requests in
        ``capture`` keep a host copy of their output (stats["captured"]):
        encryptions are copied asynchronously on their batch's stream into
        page-locked space reserved before the run (their output block is
        held until the copy has run and is not offered for replay), other
        requests synchronously."""
        be = self.be
        S = be.nstreams
        N = w.n
        if N and int(w.size.max()) > be.pool_bytes:
            raise ValueError("a request of %d bytes exceeds the %d-byte plaintext pool"
                             % (int(w.size.max()), be.pool_bytes))
        if N and ct_len(int(w.size.max())) > 1 << Arena.MAX_CLASS:
            raise ValueError("a request of %d bytes exceeds the largest arena block" % int(w.size.max()))
        # per-request state
        status = np.full(N, -1, dtype=np.int32)
        done_ms = np.full(N, np.nan)
        n_plain = w.size.copy()          # plaintext length (decrypts: that of the replayed encrypt)
        src_enc = np.full(N, -1, dtype=np.int64)  # decrypt -> encrypt it replays
        in_ref = {}                      # decrypt -> replay entry or private tampered copy
        out_blk = {}                     # request -> arena block of its output
        captured = {}
        capture = set(int(c) for c in capture)
        cap_enc = [i for i in capture if 0 <= i < N and w.kind[i] == 0]
        if cap_enc:
            be.capture_reserve(sum(ct_len(int(w.size[i])) for i in cap_enc))
        # Ciphertexts of completed encryptions, oldest first:
        # [enc, block, users, evicted, size class].  A decryption replays the
        # newest one of its own size class (else of the nearest class that has
        # one): untampered ones share it read-only, a tampered one flips a
        # byte in its own copy.  The oldest are evicted above the replay cap
        # and freed when their last user completes.
        replay = collections.deque()
        replay_cls = [collections.deque() for _ in range(NCLASS)]
        fenced = collections.deque()  # (token, blocks) released once the token is done
        replay_bytes = 0
        # Requests waiting for a slot, as a heap on (key, request): arrival
        # order ("fifo"), or arrival order within size classes with the
        # smallest class first ("small_first").
        small_first = self.policy == "small_first"
        req_cls = np.array([size_class(n) for n in w.size], dtype=np.int64)
        pending = []
        waiting_bytes = 0

        # per-request fields as Python lists (indexing numpy arrays one
        # element at a time would dominate the loop's host time)
        size_l, kind_l, tamper_l = w.size.tolist(), w.kind.tolist(), w.tamper.tolist()
        flip_l, seed_l, pwlen_l = w.flip_pos.tolist(), w.data_seed.tolist(), w.pw_len.tolist()
        cls_l = req_cls.tolist()
        pw_base = w.pw_chars.ctypes.data
        arena = self.arena
        arena_base = arena.base
        pool_base, pool_bytes = be.pool_base, be.pool_bytes

        def plain_off(i, n):
            span = pool_bytes - n
            return (seed_l[i] % span) & ~15 if span > 0 else 0

        def push(i):
            nonlocal waiting_bytes
            heapq.heappush(pending, (cls_l[i] if small_first else 0, i))
            waiting_bytes += size_l[i]

        def pick_replay(k):
            for d in range(NCLASS):
                for c in ((k + d, k - d) if d else (k,)):
                    if 0 <= c < NCLASS and replay_cls[c]:
                        return replay_cls[c][-1]
            return None
        inflight = [None] * S
        nxt = 0
        mismatches = 0
        checked = 0
        batches = 0
        launches0 = be.launch_count()
        max_batch_seen = 0

        be.start()
        cpu0 = time.process_time()
        last_arrival = float(w.t[-1]) if N else 0.0

        def unref(entry):
            entry[2] -= 1
            if entry[3] and entry[2] == 0:
                self.arena.release(entry[1])

        def evict():
            nonlocal replay_bytes
            while replay_bytes > self.replay_cap and len(replay) > 1:
                entry = replay.popleft()
                oldest = replay_cls[entry[4]].popleft()
                assert oldest is entry
                replay_bytes -= 1 << entry[1][1]
                entry[3] = True
                if entry[2] == 0:
                    self.arena.release(entry[1])

        def complete(s):
            nonlocal replay_bytes, mismatches, checked
            rec = inflight[s]
            idx = rec["idx"]
            ms = be.finish_ms(rec["token"])
            held = []
            st_a = be.statuses(s, len(idx))
            status[idx] = st_a
            done_ms[idx] = ms
            st = st_a.tolist()
            for k, i in enumerate(idx):
                if kind_l[i] == 0:
                    blk = out_blk.pop(i)
                    if i in capture:
                        # copied without waiting; the block is held until
                        # the copy has run and is not replayed
                        captured[i] = be.capture_async(s, blk, rec["out_len"][k])
                        held.append(blk)
                    elif st[k] == 0:
                        entry = [i, blk, 0, False, cls_l[i]]
                        replay.append(entry)
                        replay_cls[entry[4]].append(entry)
                        replay_bytes += 1 << blk[1]
                    else:
                        arena.release(blk)
                else:
                    if i in capture:
                        captured[i] = be.read(out_blk[i], rec["out_len"][k])
                    e = src_enc[i]
                    if st[k] == 0 and (i // 2) % verify_every == 0:
                        # compared on the device without waiting; the block
                        # is held until the comparison has run
                        n = int(n_plain[i])
                        be.verify_async(s, out_blk[i], n, plain_off(e, n))
                        checked += 1
                        held.append(out_blk.pop(i))
                    else:
                        arena.release(out_blk.pop(i))
                    ref = in_ref.pop(i)
                    if isinstance(ref, list):
                        unref(ref)
                    else:
                        arena.release(ref)
            if held:
                fenced.append((be.fence(s), held))
            evict()
            inflight[s] = None

        def release_fenced():
            while fenced and be.done(fenced[0][0]):
                for blk in fenced.popleft()[1]:
                    arena.release(blk)

        def form_batch(s):
            nonlocal waiting_bytes
            idx, out_len, rows = [], [], []
            nbytes = 0
            kept = []
            cap = self.max_batch_bytes
            if self.max_adaptive_bytes > cap and waiting_bytes > self.backlog_batches * S * cap:
                cap = min(self.max_adaptive_bytes, max(cap, waiting_bytes // S))
            limit = self.max_batch_requests
            while pending and len(idx) < limit and nbytes < cap:
                i = heapq.heappop(pending)[1]
                waiting_bytes -= size_l[i]
                if kind_l[i] == 0:
                    n = size_l[i]
                    c = n + T * (((n + B - 1) // B) or 1)
                    blk = arena.alloc(c)
                    if blk is None:
                        kept.append(i)
                        break
                    out_blk[i] = blk
                    rows.append((pw_base + 32 * i, pwlen_l[i], 0, pool_base + plain_off(i, n), n,
                                 arena_base + blk[0], c))
                    out_len.append(c)
                    nbytes += n
                else:
                    entry = pick_replay(cls_l[i])
                    if entry is None:
                        kept.append(i)
                        continue
                    e, cblk = entry[0], entry[1]
                    n = size_l[e]
                    c = n + T * (((n + B - 1) // B) or 1)
                    blk = arena.alloc(n)
                    if blk is None:
                        kept.append(i)
                        break
                    if tamper_l[i]:
                        own = arena.alloc(c)
                        if own is None:
                            arena.release(blk)
                            kept.append(i)
                            break
                        be.tamper_copy(s, own, cblk, c, flip_l[i] % c)
                        in_ref[i] = own
                        src = arena_base + own[0]
                    else:
                        entry[2] += 1
                        in_ref[i] = entry
                        src = arena_base + cblk[0]
                    out_blk[i] = blk
                    src_enc[i] = e
                    n_plain[i] = n
                    rows.append((pw_base + 32 * e, pwlen_l[e], 1, src, c, arena_base + blk[0], n))
                    out_len.append(n)
                    nbytes += n
                idx.append(i)
            if rows:
                self.reqs[s][:len(rows)] = rows
            for i in kept:
                push(i)
            return idx, out_len, nbytes

        def launch(s, idx, out_len, nbytes):
            nonlocal batches, max_batch_seen
            token = be.launch(s, self.reqs[s], len(idx))
            inflight[s] = {"idx": idx, "out_len": out_len, "token": token}
            batches += 1
            max_batch_seen = max(max_batch_seen, nbytes)

        while True:
            now = be.clock()
            progressed = False
            j = int(np.searchsorted(w.t, now, side="right"))
            if j > nxt:
                for i in range(nxt, j):
                    push(i)
                nxt = j
                progressed = True
            for s in range(S):
                if inflight[s] is not None and be.done(inflight[s]["token"]):
                    complete(s)
                    progressed = True
            release_fenced()
            for s in range(S):
                if inflight[s] is None and pending:
                    idx, out_len, nbytes = form_batch(s)
                    if idx:
                        launch(s, idx, out_len, nbytes)
                        progressed = True
            if nxt >= N and not pending and all(f is None for f in inflight):
                break
            if now > last_arrival + drain_timeout:
                break
            if not progressed:
                time.sleep(poll)
        wall = be.clock()
        host_cpu = time.process_time() - cpu0
        be.sync()
        mismatches += be.mismatches()
        # release what is still held
        release_fenced()
        for _, blks in fenced:
            for blk in blks:
                arena.release(blk)
        fenced.clear()
        for entry in replay:
            entry[3] = True
            if entry[2] == 0:
                self.arena.release(entry[1])
        replay.clear()
        for q in replay_cls:
            q.clear()

        ok = ~np.isnan(done_ms)
        lat_ms = done_ms[ok] - 1e3 * w.t[ok]
        served_bytes = int(n_plain[ok].sum())
        span_s = (np.nanmax(done_ms) / 1e3) if ok.any() else wall
        tampered = w.tamper & ok
        untampered_dec = (w.kind == 1) & ~w.tamper & ok
        return {
            "requests": int(N), "completed": int(ok.sum()),
            "p50_ms": float(np.percentile(lat_ms, 50)) if lat_ms.size else None,
            "p99_ms": float(np.percentile(lat_ms, 99)) if lat_ms.size else None,
            "mean_ms": float(lat_ms.mean()) if lat_ms.size else None,
            "served_GBps": served_bytes / span_s / 1e9,
            "offered_GBps": float(w.size.sum()) / max(1e-9, float(w.t[-1])) / 1e9 if N else 0.0,
            "duration_s": float(w.t[-1]) if N else 0.0, "wall_s": wall,
            "batches": batches,
            "gpu_launches": be.launch_count() - launches0,
            "host_cpu_s": host_cpu,
            "max_batch_bytes": max_batch_seen,
            "tampered": int(tampered.sum()),
            "tampered_rejected": int((status[tampered] == lc.LC_ERR_INTEGRITY).sum()),
            "untampered_decrypts": int(untampered_dec.sum()),
            "untampered_decrypts_ok": int((status[untampered_dec] == 0).sum()),
            "encrypts_ok": int(((w.kind == 0) & ok & (status == 0)).sum()),
            "plaintext_checked": checked, "plaintext_mismatches": mismatches,
            "arena_peak_bytes": self.arena.peak,
            "status": status, "done_ms": done_ms, "captured": captured,
            "src_enc": src_enc, "n_plain": n_plain,
        }
