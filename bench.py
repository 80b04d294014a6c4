"""Benchmark of the batched Lorenz-cipher path (one JSON line on stdout).

Workload (default): 4096 messages with log-uniform sizes in [1 KiB, 4 MiB]
(seeded), each with its own 8-32-char password; messages 0..2047 are
encrypted, 2048..4095 decrypted (their inputs are ciphertexts of seeded
plaintexts, made before timing).  One step = one lc_run_batch: host key
schedules (cached), the flattened part table, the persistent cipher kernel
and the verdict/finalize kernel, replayed from a CUDA graph.

  value   message bytes / second over K timed steps, inputs resident in HBM
  e2e     the same from pinned host buffers, host<->device copies inside the
          timed region: lc_submit_batch_host / lc_wait_batch_host with step k+1
          submitted before step k's results are read (sync_value: one
          synchronous lc_run_batch_host per step)
  roofline  the cipher kernel's FP64 operation rate against the FP64 issue
          peak (the kernel is bound by binary64 arithmetic, not HBM)
  per_message_launch  a sample of the same messages launched one per call
  cpu_baseline  the CPU oracle on the host cores, on a bounded sample

--impl reference times the CPU oracle (the only reference implementation
of this method) on a bounded sample of the same workload.

Multi-GPU (torchrun, N > 1): every rank runs its own copy of the workload
(weak scaling, no data-path collective); timing is max over ranks.
"""
import argparse
import collections
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Bit-exact encrypt/decrypt GB/s, batched vs per-message launch; served p50/p99 ms"
UNIT = "GB/s"
WORKLOAD = ("batched: 4096 messages, log-uniform 1 KiB-4 MiB, per-message 8-32-char passwords, "
            "half encrypt / half decrypt, parallel mode (4096-byte parts), one persistent launch "
            "from a CUDA graph per step")
NOMINAL_FP64_TFLOPS = 1.25  # recipe: GB300 dense FP64, counting a DFMA as 2 flops


# ---------------------------------------------------------------------------
# distributed helpers (CPU-testable with gloo)
# ---------------------------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(backend):
    import torch.distributed as dist
    ws, rank, _ = dist_env()
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=ws)
    return ws, rank


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def workload_spec(count):
    from paper_1201_3114_gb300 import synth
    return synth.cfg4_spec(count=count)


def fp64_ops_per_launch(sizes, n_warm=3000, steps=1, B=4096, T=8):
    """Algorithmic binary64 operations (each DADD/DMUL one operation, no FMA)
    of one launch over messages of these plaintext sizes, and the bytes each
    trajectory handles: per part 15 n_warm (warm-up) + 4 (start point)
    + 3 (first alpha scaling), per byte (body and tag) 15 S (Euler) + 1 (kick)
    + 3 (alpha scaling) + 3 (r += a')."""
    sizes = np.asarray(sizes, dtype=np.int64)
    parts = np.maximum(1, -(-sizes // B))
    traj_bytes = sizes + T * parts
    per_part = 15 * n_warm + 4 + 3
    per_byte = 15 * steps + 1 + 3 + 3
    ops = int(parts.sum()) * per_part + int(traj_bytes.sum()) * per_byte
    return ops, int(parts.sum()), int(traj_bytes.sum())


def fp64_pipe_ops_per_launch(sizes, mask, n_warm=3000, steps=1, B=4096, T=8, warm_mask=None):
    """Binary64 operations of one launch that run on the FP64 pipe when the
    kernel computes the operations selected by `mask` (lc_emu_mask; the
    warm-up's Euler steps by `warm_mask`, lc_warm_mask) with exact integer
    arithmetic: the Euler step keeps 15 minus its emulated operations, each
    byte also has the kick, r += a' (3) and, after the (mu, Omega) lock, one
    alpha scaling; each part 4 seeding operations."""
    sizes = np.asarray(sizes, dtype=np.int64)
    parts = np.maximum(1, -(-sizes // B))
    traj_bytes = sizes + T * parts

    def euler_hw(m):
        return 15 - (2 * (m & 1) + bin(m & 0x7FFC).count("1"))

    wm = mask if warm_mask is None else warm_mask
    per_byte = steps * euler_hw(mask) + (0 if mask & (1 << 15) else 1) + (0 if mask & (1 << 16) else 3) \
        + (0 if mask & 2 else 1)
    per_part = n_warm * euler_hw(wm) + 4
    return int(parts.sum()) * per_part + int(traj_bytes.sum()) * per_byte


# the sources the cipher kernel's code comes from (of include/lc.h it takes
# only the values of two status codes)
KERNEL_SOURCES = ("paper_1201_3114_gb300/csrc/cipher.cu", "paper_1201_3114_gb300/csrc/softfp64.cuh",
                  "paper_1201_3114_gb300/csrc/lc_internal.h")


def source_hash():
    """Hash of the cipher kernel's sources (keys the committed ncu traffic)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(os.path.basename(f).encode() + fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    """The measured HBM copy and bf16 GEMM peaks of this GPU model, if recorded."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def committed_traffic(dense_build=0):
    """DRAM bytes and warp instructions per message byte of the throughput
    variant's build (the default one, or the dense one when dense_build) from
    the committed ncu summary, if it was taken on the current kernel
    sources."""
    path = os.path.join(ROOT, "profiles", "batch_kernel_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != source_hash():
        return None
    return rec.get("builds", {}).get("dense" if dense_build else "default")


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample_plan(spec, target_bytes):
    """(message, first part, parts) triples covering ~target_bytes, spread
    over all messages in proportion to their size."""
    sizes = spec["sizes"]
    total = int(sizes.sum())
    frac = min(1.0, target_bytes / max(1, total))
    plan = []
    for m, n in enumerate(sizes):
        nb = max(1, -(-int(n) // 4096))
        take = max(1, int(round(nb * frac)))
        plan.append((m, 0, min(nb, take)))
    return plan


def run_oracle_sample(spec, plan, threads):
    """Run the sampled parts through the oracle on `threads` host threads.
    Returns (message bytes processed, wall seconds)."""
    import oracle as O
    from paper_1201_3114_gb300 import synth
    prm = O.params()
    jobs = []
    for m, b0, nb in plan:
        n = int(spec["sizes"][m])
        key = O.key_schedule(spec["pws"][m], prm)
        lo, hi = b0 * 4096, min(n, (b0 + nb) * 4096)
        P = np.zeros(n, dtype=np.uint8)
        P[lo:hi] = synth.uniform_bytes(spec["data_seeds"][m], hi - lo, lo)
        Cb = np.zeros(O.ciphertext_len(n, O.PARALLEL, prm), dtype=np.uint8)
        jobs.append((spec["dirs"][m], key, P, n, Cb, b0, b0 + nb, hi - lo))
    done = []
    lock = threading.Lock()
    it = iter(jobs)

    def worker():
        while True:
            with lock:
                job = next(it, None)
            if job is None:
                return
            d, key, P, n, Cb, b0, b1, nbytes = job
            if d == 0:
                O.encrypt_blocks(key, P, n, Cb, b0, b1, prm)
            else:
                O.decrypt_blocks(key, Cb, n, P, b0, b1, prm)
            with lock:
                done.append(nbytes)

    t0 = time.perf_counter()
    ths = [threading.Thread(target=worker) for _ in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    return int(sum(done)), time.perf_counter() - t0


def reference_arm(args):
    """The CPU oracle timed on the host cores, on a bounded sample of the
    workload per step (rank 0 only)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    spec = workload_spec(args.messages)
    threads = os.cpu_count() or 1
    plan = oracle_sample_plan(spec, args.ref_sample_mb << 20)
    for _ in range(args.warmup):
        run_oracle_sample(spec, plan, threads)
    tot_b, tot_s = 0, 0.0
    for _ in range(args.steps):
        b, s = run_oracle_sample(spec, plan, threads)
        tot_b += b
        tot_s += s
    v = tot_b / tot_s / 1e9
    sample = "%d MiB of parts per step spread over all %d messages (first parts of each)" % (
        tot_b // args.steps >> 20, len(spec["sizes"]))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "messages": len(spec["sizes"]), "mode": "parallel",
                   "sample": sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_serving(seconds, rate, device, capacity_gbps, policy="small_first", max_batch_mib=128,
                low_seconds=15.0, capture_per_class=125, streams=6):
    """The served configuration (Poisson arrivals, log-uniform 256 B - 16 MiB,
    50/50, 2 % tampered decrypts, 48 GiB admission budget) for `seconds` of
    arrivals, then a supplementary run of `low_seconds` at 0.8x the measured
    batched capacity, labelled as such.  In the first run a seeded sample of
    encryptions, up to `capture_per_class` per power-of-two size class, keeps
    a host copy of its ciphertext (copied asynchronously on the batch's
    stream); returns (records, sample) where sample lists each captured
    request's password, plaintext location in the seeded pool and output."""
    from paper_1201_3114_gb300 import serve, synth
    srv = serve.Server(device, streams=streams, budget_bytes=48 << 30, pool_bytes=1 << 30,
                       max_batch_bytes=max_batch_mib << 20, policy=policy)
    out = {}
    sample = None
    try:
        for label, r, secs in (("offered", rate, seconds), ("at_0.8x_capacity", None, low_seconds)):
            if secs <= 0:
                continue
            if r is None:
                mean = 1.5e6
                r = 0.8 * capacity_gbps * 1e9 / mean
            w = serve.Workload(synth.cfg5_spec(rate=r, duration=secs))
            cap = serve.capture_sample(w, capture_per_class) if (label == "offered" and
                                                                 capture_per_class) else []
            st = srv.run(w, capture=cap)
            keep = ("requests", "completed", "p50_ms", "p99_ms", "mean_ms", "served_GBps",
                    "offered_GBps", "duration_s", "wall_s", "batches", "gpu_launches", "tampered",
                    "tampered_rejected", "untampered_decrypts", "untampered_decrypts_ok",
                    "encrypts_ok", "plaintext_checked", "plaintext_mismatches", "max_batch_bytes")
            rec = {k: st[k] for k in keep}
            rec["policy"] = policy
            rec["streams"] = streams
            rec["rate_req_per_s"] = r
            rec["served_over_per_message"] = None
            out[label] = rec
            if cap:
                sample = {"pool_seed": srv.be.pool_seed, "label": label,
                          "items": [(w.pw(i), int(w.size[i]), srv.plain_offset(w, i, int(w.size[i])),
                                     st["captured"][i]) for i in cap]}
    finally:
        srv.close()
    return out, sample


def oracle_config_rates(threads, cfg3_mib=256):
    """The oracle timed on the single-message configurations: 64 KiB and the
    1 MiB text (parallel mode on one core and on all cores, sequential mode on
    one core: it is one trajectory), and a sample of the 1 GiB message (its
    first cfg3_mib MiB, all cores).  Message bytes per second, decimal GB."""
    import oracle as O
    from concurrent.futures import ThreadPoolExecutor
    from paper_1201_3114_gb300 import synth
    prm = O.params()

    def par(pw, P, nthreads):
        key = O.key_schedule(pw, prm)
        n = P.size
        nb = max(1, -(-n // 4096))
        Cb = np.zeros(O.ciphertext_len(n, O.PARALLEL, prm), dtype=np.uint8)
        step = max(1, min(64, -(-nb // nthreads)))
        jobs = [(b, min(nb, b + step)) for b in range(0, nb, step)]
        with ThreadPoolExecutor(nthreads) as ex:
            list(ex.map(lambda _: None, range(4 * nthreads)))  # threads started before timing
            t0 = time.perf_counter()
            list(ex.map(lambda j: O.encrypt_blocks(key, P, n, Cb, j[0], j[1], prm), jobs))
            secs = time.perf_counter() - t0
        return n / secs / 1e9

    out = {}
    c1 = synth.cfg1()
    out["cfg1_64k"] = {"one_core_GBps": par(c1["pw"], c1["P"], 1),
                       "all_cores_GBps": par(c1["pw"], c1["P"], threads)}
    c2 = synth.cfg2()
    t0 = time.perf_counter()
    O.encrypt(c2["pw"], c2["P"], O.SEQUENTIAL, prm)
    seq = c2["P"].size / (time.perf_counter() - t0) / 1e9
    out["cfg2_1mib"] = {"parallel_one_core_GBps": par(c2["pw"], c2["P"], 1),
                        "parallel_all_cores_GBps": par(c2["pw"], c2["P"], threads),
                        "sequential_one_core_GBps": seq}
    spec = synth.cfg3_spec()
    n3 = cfg3_mib << 20
    P3 = np.empty(n3, dtype=np.uint8)
    chunk = 16 << 20

    def fill(a):
        P3[a:a + chunk] = synth.uniform_bytes(spec["data_seed"], min(chunk, n3 - a), a)

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(fill, range(0, n3, chunk)))
    out["cfg3_1gib"] = {"all_cores_GBps": par(spec["pw"], P3, threads),
                        "sample": "the first %d MiB of the 1 GiB message" % cfg3_mib}
    out["cores"] = threads
    return out


def oracle_check_served(sample, threads):
    """CPU-baseline leg for the served configuration: the oracle encrypts the
    captured sample (plaintexts regenerated on the host from the pool's
    seed) on `threads` host threads; returns the oracle's rate and how many
    served ciphertexts differ from it."""
    import oracle as O
    from concurrent.futures import ThreadPoolExecutor
    from paper_1201_3114_gb300 import synth
    prm = O.params()
    items = sample["items"]
    plains = [None] * len(items)

    def gen(k):
        _, n, off, _ = items[k]
        plains[k] = synth.uniform_bytes(sample["pool_seed"], n, off)

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(gen, range(len(items))))
    keys = [O.key_schedule(pw, prm) for pw, _, _, _ in items]
    outs = [np.zeros(O.ciphertext_len(n, O.PARALLEL, prm), dtype=np.uint8) for _, n, _, _ in items]
    jobs = []
    for k, (_, n, _, _) in enumerate(items):
        nb = max(1, -(-n // 4096))
        jobs += [(k, b, min(nb, b + 64)) for b in range(0, nb, 64)]
    jobs.sort(key=lambda j: -items[j[0]][1])

    def run(job):
        k, b0, b1 = job
        O.encrypt_blocks(keys[k], plains[k], plains[k].size, outs[k], b0, b1, prm)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(run, jobs))
    secs = time.perf_counter() - t0
    nbytes = sum(n for _, n, _, _ in items)
    bad = sum(1 for k, it in enumerate(items) if not np.array_equal(it[3], outs[k]))
    return {"value": nbytes / secs / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d captured encryptions of the served run, every size class 256 B - 16 MiB "
                      "(%.0f MiB)" % (len(items), nbytes / 2 ** 20),
            "wall_s": secs}, len(items), bad


def single_message_configs(ctx, dev, stream, pipes, sm_mhz, reps=20):
    """The single-message configurations, through lc_encrypt / lc_decrypt on
    device-resident buffers (CUDA events on the launching stream; lc_decrypt
    synchronises, so its times include the verdict read-back):

      cfg1_64k   64 KiB uniform bytes, 16-char password, parallel mode
      cfg2_1mib  1 MiB Zipf text with a 4 KiB zero run, 32-char password, both
                 modes; one flipped ciphertext byte must be rejected
      cfg3_1gib  1 GiB uniform bytes, 24-char password, parallel mode, with
                 the cipher kernel's time, its binary64 rate and roofline
                 fractions

    Round trips are checked here; bit-exactness against the oracle is the
    parity tests' job (tests/test_gpu_parity.py)."""
    import torch
    from paper_1201_3114_gb300 import lc, synth

    def ev_time(fn, n):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    def enc_dec(pw, P, mode, n_rep, n_warm=3):
        n = P.numel()
        C = torch.empty(ctx.ciphertext_len(n, mode), dtype=torch.uint8, device=dev)
        back = torch.empty(max(1, n), dtype=torch.uint8, device=dev)
        enc = lambda: lc.check(lc.lc_encrypt(ctx.handle, pw, P, n, C, C.numel(), mode, stream))
        dec = lambda: lc.check(lc.lc_decrypt(ctx.handle, pw, C, C.numel(), back, n, mode, stream))
        for _ in range(n_warm):
            enc()
            dec()
        ms_e = ev_time(enc, n_rep)
        ms_d = ev_time(dec, n_rep)
        if not torch.equal(back[:n], P):
            raise SystemExit("round trip failed (mode %d, %d bytes)" % (mode, n))
        return C, ms_e, ms_d

    out = {}
    c1 = synth.cfg1()
    P1 = torch.from_numpy(c1["P"]).to(dev)
    _, me, md = enc_dec(c1["pw"], P1, lc.LC_PARALLEL, reps)
    n1 = P1.numel()
    out["cfg1_64k"] = {"bytes": n1, "parts": n1 // 4096, "encrypt_ms": me, "decrypt_ms": md,
                       "encrypt_GBps": n1 / me / 1e6, "decrypt_GBps": n1 / md / 1e6,
                       "note": "16 parts: one part's serial chain (3000 warm-up + 4104 byte steps) "
                               "sets the latency"}
    c2 = synth.cfg2()
    P2 = torch.from_numpy(c2["P"]).to(dev)
    n2 = P2.numel()
    rec = {"bytes": n2}
    for mode, name, nrep, nwarm in ((lc.LC_PARALLEL, "parallel", reps, 3),
                                    (lc.LC_SEQUENTIAL, "sequential", 2, 1)):
        C2, me, md = enc_dec(c2["pw"], P2, mode, nrep, nwarm)
        bad = C2.clone()
        pos = synth.word(c2["flip_seed"], mode) % bad.numel()
        bad[pos] ^= 1 + synth.word(c2["flip_seed"], 10 + mode) % 255
        st, _ = ctx.decrypt(c2["pw"], bad, mode)
        rec[name] = {"encrypt_ms": me, "decrypt_ms": md, "encrypt_GBps": n2 / me / 1e6,
                     "decrypt_GBps": n2 / md / 1e6,
                     "flipped_byte_rejected": st == lc.LC_ERR_INTEGRITY}
        if st != lc.LC_ERR_INTEGRITY:
            raise SystemExit("config 2: a flipped ciphertext byte was accepted (mode %d)" % mode)
    rec["parallel_over_sequential"] = rec["parallel"]["encrypt_GBps"] / rec["sequential"]["encrypt_GBps"]
    out["cfg2_1mib"] = rec
    del P1, P2

    spec = synth.cfg3_spec()
    n3, pw3 = spec["n"], spec["pw"]
    P3 = torch.empty(n3, dtype=torch.uint8, device=dev)
    lc.check(lc.lc_synth_uniform(P3, n3, spec["data_seed"], 0, stream))
    C3 = torch.empty(ctx.ciphertext_len(n3), dtype=torch.uint8, device=dev)
    enc3 = lambda: lc.check(lc.lc_encrypt(ctx.handle, pw3, P3, n3, C3, C3.numel(), lc.LC_PARALLEL, stream))
    for _ in range(3):
        enc3()
    lc.check(lc.lc_ctx_timing(ctx.handle, True))
    ms = ev_time(enc3, 5)
    kms, kn = lc.lc_ctx_kernel_time(ctx.handle)
    lc.check(lc.lc_ctx_timing(ctx.handle, False))
    kms = kms / max(1, kn)
    st, back = ctx.decrypt(pw3, C3)
    if st != lc.LC_OK or not torch.equal(back, P3):
        raise SystemExit("config 3: round trip failed")
    del back
    sizes = [n3]
    ops, parts, _ = fp64_ops_per_launch(sizes)
    rl = roofline_terms(sizes, kms, pipes, sm_mhz, dense_build=lc.lc_ctx_get_launch(ctx.handle).dense_build)
    out["cfg3_1gib"] = {"bytes": n3, "parts": parts, "ms_per_encrypt": ms, "GBps": n3 / ms / 1e6,
                        "kernel_ms": kms, "kernel_GBps": n3 / kms / 1e6,
                        "fp64_ops_per_launch": ops, "fp64_gops": ops / (kms * 1e-3) / 1e9,
                        "method_roofline_GBps": rl["method_roofline_GBps"],
                        "method_roofline_frac": (n3 / kms / 1e6) / rl["method_roofline_GBps"],
                        "fp64_pipe_frac_of_probe": rl["fp64_pipe_frac_of_probe"],
                        "joint": rl["joint"]}
    del P3, C3
    torch.cuda.empty_cache()
    return out


def roofline_terms(sizes, kernel_ms, pipes, sm_mhz, n_warm=3000, steps=1, B=4096, T=8, dense_build=0):
    """Roofline figures of one cipher-kernel launch over messages of these
    sizes:
      method_roofline_GBps  the bound the method statement names: the slower of
                the binary64 arithmetic at the nominal FP64 peak (33 operations
                per byte, warm-up included) and 2 bytes per byte at HBM speed
      fp64_pipe_*  the binary64 operations that run on the FP64 pipe against
                the probed DADD rate
      joint     the kernel's own ceiling: the FP64-pipe time of those
                operations at the probed rate, and the issue time of its
                instructions (the committed ncu count per message byte, on the
                same kernel sources) at 4 warp-instructions per SM per clock;
                frac = the larger of the two over the measured kernel time"""
    from paper_1201_3114_gb300 import lc
    ops, parts, traj = fp64_ops_per_launch(sizes, n_warm, steps, B, T)
    msg_bytes = int(np.asarray(sizes, dtype=np.int64).sum())
    peak_slot = NOMINAL_FP64_TFLOPS * 1e3 / 2.0
    hbm = measured_peaks().get("hbm_gbs") or 6800.0
    per_byte = ops / max(1, msg_bytes)
    method_gbps = min(peak_slot / per_byte, hbm / (2.0 + 8.0 * parts / max(1, msg_bytes)))
    mask = lc.lc_emu_mask()
    hw_ops = fp64_pipe_ops_per_launch(sizes, mask, n_warm, steps, B, T, lc.lc_warm_mask())
    t_fp64 = hw_ops / (pipes.dadd_gops * 1e9) * 1e3
    rec = committed_traffic(dense_build)
    joint = None
    if rec and rec.get("inst_executed_per_message_byte") and sm_mhz:
        inst = rec["inst_executed_per_message_byte"] * msg_bytes
        t_issue = inst / (pipes.sm_count * 4 * sm_mhz * 1e6) * 1e3
        bound = max(t_fp64, t_issue)
        joint = {"fp64_pipe_ms": t_fp64, "issue_ms": t_issue, "kernel_ms": kernel_ms,
                 "bound": "fp64_pipe" if t_fp64 >= t_issue else "issue",
                 "frac": bound / kernel_ms,
                 "fp64_pipe_ops": hw_ops, "fp64_pipe_rate_gops": pipes.dadd_gops,
                 "warp_instructions": inst, "sm_count": pipes.sm_count, "sm_mhz": sm_mhz,
                 "build": "dense" if dense_build else "default",
                 "note": "warp instructions scaled from the committed ncu count per message byte "
                         "of the same build (profiles/batch_kernel_traffic.json, same kernel sources)"}
    return {"method_roofline_GBps": method_gbps,
            "fp64_pipe_frac_of_probe": (hw_ops / (kernel_ms * 1e-3) / 1e9) / pipes.dadd_gops,
            "joint": joint}


def profile_case(args):
    """One message of args.profile_case MiB, parallel-mode encryption per step."""
    import torch
    from paper_1201_3114_gb300 import lc
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n = args.profile_case << 20
    ctx = lc.Context(0)
    P = torch.empty(n, dtype=torch.uint8, device="cuda")
    lc.check(lc.lc_synth_uniform(P, n, 0x1201311400CA5E, 0, stream))
    Cb = torch.empty(ctx.ciphertext_len(n), dtype=torch.uint8, device="cuda")
    pw = b"profile-case-24-chars-pw"
    # the throughput variant's full-grid build, whatever the case's size
    l = lc.lc_ctx_get_launch(ctx.handle)
    if args.profile_launch:
        l.threads_per_cta, l.dense_build = (int(v) for v in args.profile_launch.split(","))
    lc.check(lc.lc_ctx_set_launch(ctx.handle, l.threads_per_cta, l.ctas_per_sm, l.smem_staging,
                                  l.small_batch_rows, l.host_chunk_mib, l.dense_build, 1))
    for _ in range(args.warmup):
        lc.check(lc.lc_encrypt(ctx.handle, pw, P, n, Cb, Cb.numel(), lc.LC_PARALLEL, stream))
    lc.check(lc.lc_ctx_timing(ctx.handle, True))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        lc.check(lc.lc_encrypt(ctx.handle, pw, P, n, Cb, Cb.numel(), lc.LC_PARALLEL, stream))
    e1.record(stream)
    torch.cuda.synchronize()
    kms, kn = lc.lc_ctx_kernel_time(ctx.handle)
    ops, parts, _ = fp64_ops_per_launch([n])
    ms = e0.elapsed_time(e1) / args.steps
    # one statistics pass over the ciphertext (outside the timed region)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    st = lc.lc_byte_stats(ctx.handle, Cb, n, 8, stream)
    s1.record(stream)
    torch.cuda.synchronize()
    stats_ms = s0.elapsed_time(s1)
    # and one histogram-only pass (the direct kernel)
    s0.record(stream)
    lc.lc_byte_stats(ctx.handle, Cb, n, 0, stream)
    s1.record(stream)
    torch.cuda.synchronize()
    hist_ms = s0.elapsed_time(s1)
    print(json.dumps({"case": "profile", "mib": args.profile_case, "ms_per_step": ms,
                      "GBps": n / ms / 1e6, "kernel_ms": kms / max(1, kn),
                      "fp64_gops": ops / (kms / max(1, kn)) / 1e6, "source_hash": source_hash(),
                      "stats_ms": stats_ms, "stats_GBps": n / stats_ms / 1e6,
                      "histogram_ms": hist_ms, "histogram_GBps": n / hist_ms / 1e6,
                      "launch": lc.lc_ctx_get_launch(ctx.handle).as_dict(),
                      "ciphertext_entropy_bits": lc.entropy_bits(st)}))
    ctx.close()
    return 0


def latency_case(args):
    """One parallel-mode encryption of args.latency_case KiB per step with the
    FP64-pipe variant: the split build (each part's coordinates on three
    warps, the default for small batches) and the one-part-per-thread build."""
    import torch
    from paper_1201_3114_gb300 import lc, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n = args.latency_case << 10
    P = torch.from_numpy(synth.uniform_bytes(synth.config_seed(1) + 30, n)).cuda()
    out = {"case": "latency", "kib": args.latency_case, "parts": -(-n // 4096), "source_hash": source_hash()}
    with lc.Context(0) as ctx:
        for name, split in (("three_warps", 0xFFFFFFFF), ("one_thread", 1)):
            lc.check(lc.lc_ctx_set_launch(ctx.handle, 256, 0, 0, 0xFFFFFFFF, 0, 0, 0, split))
            enc = lambda: ctx.encrypt(b"latency-case-password", P, stream=stream)
            for _ in range(args.warmup):
                enc()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                enc()
            e1.record(stream)
            torch.cuda.synchronize()
            out[name + "_ms"] = e0.elapsed_time(e1) / args.steps
    print(json.dumps(out))
    return 0


def next_rows(args):
    """Throughput of the widened rows: batched sequential mode (one message
    per thread), the S = 3000 steps-per-byte profile, the delta t = 0.027
    profile and the ciphertext statistics kernel.  One JSON line."""
    import torch
    from paper_1201_3114_gb300 import lc, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = {"case": "next_rows", "source_hash": source_hash()}

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def check_status(st):
        bad = int((st != 0).sum())
        if bad:
            raise SystemExit("next_rows: %d requests failed" % bad)

    # batched sequential mode: one 16 KiB message per resident thread of
    # the persistent grid (3 CTAs x 256 threads per SM), against the same
    # messages in parallel mode (4 parts each)
    with lc.Context(0) as ctx:
        cnt, sz = sms * 768, 16384
        arena = torch.empty(cnt * sz, dtype=torch.uint8, device="cuda")
        lc.check(lc.lc_synth_uniform(arena, cnt * sz, synth.config_seed(3) + 17, 0, stream))
        res = {}
        for mode, name in ((lc.LC_SEQUENTIAL, "sequential"), (lc.LC_PARALLEL, "parallel")):
            clen = ctx.ciphertext_len(sz, mode)
            outb = torch.empty(cnt * clen, dtype=torch.uint8, device="cuda")
            pws = [synth.password(synth.subseed(synth.config_seed(3), 5000 + i), 16) for i in range(256)]
            items = [(pws[i % 256], lc.LC_ENCRYPT, arena.data_ptr() + i * sz, sz,
                      outb.data_ptr() + i * clen, clen) for i in range(cnt)]
            b = lc.Batch(items)
            st = torch.full((cnt,), -1, dtype=torch.int32, device="cuda")
            ms = timed(lambda: lc.check(lc.lc_run_batch(ctx.handle, b, st, mode, stream)), args.steps)
            check_status(st)
            res[name] = {"ms_per_batch": ms, "GBps": cnt * sz / ms / 1e6}
            del outb
        out["batched_sequential"] = {
            "messages": cnt, "message_bytes": sz, **{k: v for k, v in res.items()},
            "sequential_over_parallel": res["sequential"]["GBps"] / res["parallel"]["GBps"],
            "note": "sequential: one trajectory of 16384 + 8 steps and one warm-up per message; "
                    "parallel: 4 parts, each with its own warm-up"}
        del arena

    # the S = 3000 profile (one Euler step count per byte read as n_it):
    # 64-byte parts, one part per resident thread
    with lc.Context(0, lc.params(steps_per_byte=3000, block_len=64)) as c:
        n = sms * 768 * 64
        P = torch.empty(n, dtype=torch.uint8, device="cuda")
        lc.check(lc.lc_synth_uniform(P, n, synth.config_seed(3) + 18, 0, stream))
        Cb = torch.empty(c.ciphertext_len(n), dtype=torch.uint8, device="cuda")
        ms = timed(lambda: lc.check(lc.lc_encrypt(c.handle, b"n_it-profile-pw", P, n, Cb, Cb.numel(),
                                                  lc.LC_PARALLEL, stream)), 1)
        parts = n // 64
        steps = parts * (3000 + (64 + 8) * 3000)  # warm-up, then S steps per body and tag byte
        out["s3000_profile"] = {"bytes": n, "block_len": 64, "ms": ms, "MBps": n / ms / 1e3,
                                "euler_steps_per_s": steps / (ms * 1e-3)}

    # per-request keys (row f2): 128 messages of 4 MiB (131,072 parts) whose
    # requests carry their own k, against the same batch with the context's
    # k = (4, 4, 4), and against the general path (small-batch threshold
    # raised above the batch)
    with lc.Context(0) as c:
        nm, mb = 128, 4 << 20
        P = torch.empty(nm * mb, dtype=torch.uint8, device="cuda")
        lc.check(lc.lc_synth_uniform(P, P.numel(), synth.config_seed(4) + 23, 0, stream))
        clen = c.ciphertext_len(mb)
        Cb = torch.empty(nm * clen, dtype=torch.uint8, device="cuda")
        st = torch.empty(nm, dtype=torch.int32, device="cuda")
        ks = [(3, 4, 3), (3, 3, 3), (4, 3, 4), (4, 4, 4)]

        def items(own_k):
            return [(synth.password(synth.subseed(93, m), 8 + m % 25), 0, P.data_ptr() + m * mb, mb,
                     Cb.data_ptr() + m * clen, clen, None, ks[m % 4] if own_k else None) for m in range(nm)]

        rows = {}
        for label, own_k, small in (("context_k", False, 0), ("own_k", True, 0),
                                    ("own_k_general_path", True, 0xFFFFFFFF)):
            lc.check(lc.lc_ctx_set_launch(c.handle, 256, 0, 0, small, 0, 1))
            b = lc.BatchEx(items(own_k))
            ms = timed(lambda: lc.check(lc.lc_run_batch_ex(c.handle, b, st, lc.LC_PARALLEL, stream)), 3)
            assert int(st.max()) == 0 and int(st.min()) == 0
            rows[label] = {"ms": ms, "GBps": nm * mb / ms / 1e6}
        out["per_request_k_batched"] = dict(rows, messages=nm, message_bytes=mb,
                                            keys="k in (3,4,3), (3,3,3), (4,3,4), (4,4,4) in rotation")

    # the delta t = 0.027 profile (the trajectory leaves the attractor and
    # saturates; every emulated operation then takes its hardware fallback)
    with lc.Context(0, lc.params(dt=0.027)) as c:
        n = 256 << 20
        P = torch.empty(n, dtype=torch.uint8, device="cuda")
        lc.check(lc.lc_synth_uniform(P, n, synth.config_seed(3) + 19, 0, stream))
        Cb = torch.empty(c.ciphertext_len(n), dtype=torch.uint8, device="cuda")
        ms = timed(lambda: lc.check(lc.lc_encrypt(c.handle, b"dt-0.027-profile", P, n, Cb, Cb.numel(),
                                                  lc.LC_PARALLEL, stream)), 2)
        out["dt0027_profile"] = {"bytes": n, "ms": ms, "GBps": n / ms / 1e6}

    # ciphertext statistics (histogram, sums, lagged products) over 1 GiB
    with lc.Context(0) as ctx:
        n = 1 << 30
        P = torch.empty(n, dtype=torch.uint8, device="cuda")
        lc.check(lc.lc_synth_uniform(P, n, synth.config_seed(3) + 20, 0, stream))
        peak = measured_peaks().get("hbm_gbs")
        for lags, key in ((8, "stats_1GiB"), (0, "stats_1GiB_histogram_only")):
            ms = timed(lambda: lc.lc_byte_stats(ctx.handle, P, n, lags, stream), args.steps)
            out[key] = {"max_lag": lags, "ms": ms, "GBps": n / ms / 1e6, "hbm_peak_GBps": peak,
                        "frac_of_measured_hbm": (n / ms / 1e6) / peak if peak else None,
                        "note": "synchronous call: memset, kernel, read-back of the counters"}

        # the same statistics fused into the cipher kernel: a 1 GiB
        # encryption with counting on, against the plain encryption followed
        # by the separate pass over its ciphertext
        Cb = torch.empty(ctx.ciphertext_len(n), dtype=torch.uint8, device="cuda")
        pw = b"fused-statistics-24chars"
        enc = lambda: lc.check(lc.lc_encrypt(ctx.handle, pw, P, n, Cb, Cb.numel(), lc.LC_PARALLEL, stream))
        ms_plain = timed(enc, args.steps)
        ms_pass = timed(lambda: lc.lc_byte_stats(ctx.handle, Cb, Cb.numel(), 8, stream), args.steps)
        lc.check(lc.lc_ctx_ciphertext_stats(ctx.handle, True))
        ms_fused = timed(enc, args.steps)
        fused = lc.lc_ctx_get_ciphertext_stats(ctx.handle)
        lc.check(lc.lc_ctx_ciphertext_stats(ctx.handle, False))
        sep = lc.lc_byte_stats(ctx.handle, Cb, Cb.numel(), 8, stream)
        reps = args.warmup + args.steps
        same = (fused.n == reps * sep.n and list(fused.hist) == [reps * h for h in sep.hist]
                and list(fused.lag_sum) == [reps * v for v in sep.lag_sum])
        if not same:
            raise SystemExit("fused ciphertext statistics differ from the separate pass")
        out["stats_fused_1GiB"] = {
            "encrypt_ms": ms_plain, "encrypt_counting_ms": ms_fused, "separate_pass_ms": ms_pass,
            "fused_overhead_ms": ms_fused - ms_plain,
            "fused_overhead_frac": (ms_fused - ms_plain) / ms_plain,
            "separate_pass_frac": ms_pass / ms_plain, "equal_to_separate_pass": same}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--messages", type=int, default=4096)
    ap.add_argument("--per-message-sample", type=int, default=256)
    ap.add_argument("--cpu-sample-mb", type=int, default=512)
    ap.add_argument("--ref-sample-mb", type=int, default=96)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (lc_tune) and time the default launch shape")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the served-workload run (0 = skip); 60 s is the configuration")
    ap.add_argument("--serve-low-seconds", type=float, default=15.0,
                    help="length of the supplementary served run at 0.8x capacity (0 = skip)")
    ap.add_argument("--serve-capture", type=int, default=125,
                    help="served encryptions per size class whose ciphertexts the CPU-baseline leg "
                         "checks against the oracle (0 = none)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the single-message configurations (64 KiB, 1 MiB, 1 GiB)")
    ap.add_argument("--serve-rate", type=float, default=20000.0)
    ap.add_argument("--serve-policy", default="small_first", choices=["small_first", "fifo"],
                    help="order in which waiting requests fill a batch")
    ap.add_argument("--serve-batch-mib", type=int, default=128, help="bytes per served batch (cap)")
    ap.add_argument("--serve-streams", type=int, default=6, help="stream slots of the server")
    ap.add_argument("--profile-launch", default="", metavar="THREADS,DENSE",
                    help="--profile-case: threads per CTA and dense build of the cipher kernel "
                         "(default: the context's default launch shape; the case always runs the "
                         "full-grid build of the throughput variant)")
    ap.add_argument("--profile-case", type=int, default=0, metavar="MIB",
                    help="only time one MIB-MiB parallel-mode encryption per step (a small "
                         "case for ncu captures); prints a short JSON line")
    ap.add_argument("--latency-case", type=int, default=0, metavar="KIB",
                    help="time one small message with both FP64-pipe builds (one JSON line)")
    ap.add_argument("--next-rows", action="store_true",
                    help="only time the widened rows (batched sequential mode, the S = 3000 "
                         "and delta t = 0.027 profiles, the statistics kernel); one JSON line")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    if args.impl == "reference":
        return reference_arm(args)
    if args.profile_case:
        return profile_case(args)
    if args.latency_case:
        return latency_case(args)
    if args.next_rows:
        return next_rows(args)

    import torch
    from paper_1201_3114_gb300 import lc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    init_dist("nccl" if ws > 1 else "gloo")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    spec = workload_spec(args.messages)
    sizes, pws, seeds, dirs = spec["sizes"], spec["pws"], spec["data_seeds"], spec["dirs"]
    count = len(sizes)
    ctx = lc.Context(local)
    default_launch = lc.lc_ctx_get_launch(ctx.handle).as_dict()
    tuning = None
    if not args.no_tune:
        # tuned on a probe batch of the workload's shape and size
        t0 = time.perf_counter()
        lc.lc_tune(ctx.handle, int(sizes.sum()), stream)
        tuning = {"default": default_launch, "seconds": time.perf_counter() - t0,
                  "candidates": [dict(l, median_ms=ms) for l, ms in lc.lc_tune_report(ctx.handle)]}
    launch = lc.lc_ctx_get_launch(ctx.handle)

    # ---- device arenas: plaintexts, ciphertexts (decrypt inputs), outputs
    def aligned(v):
        return (v + 255) & ~255

    p_off, c_off, o_off = [], [], []
    ptot = ctot = otot = 0
    clen = [ctx.ciphertext_len(int(n)) for n in sizes]
    for m in range(count):
        p_off.append(ptot)
        ptot = aligned(ptot + int(sizes[m]))
        c_off.append(ctot)
        ctot = aligned(ctot + (clen[m] if dirs[m] == 1 else 0))
        o_off.append(otot)
        otot = aligned(otot + (clen[m] if dirs[m] == 0 else int(sizes[m])))
    Parena = torch.empty(ptot, dtype=torch.uint8, device=dev)
    Carena = torch.empty(max(ctot, 256), dtype=torch.uint8, device=dev)
    Oarena = torch.empty(otot, dtype=torch.uint8, device=dev)
    for m in range(count):
        lc.check(lc.lc_synth_uniform(Parena.data_ptr() + p_off[m], int(sizes[m]), seeds[m], 0, stream))
    enc_items = [(pws[m], 0, Parena.data_ptr() + p_off[m], int(sizes[m]),
                  Carena.data_ptr() + c_off[m], clen[m]) for m in range(count) if dirs[m] == 1]
    st_setup = torch.zeros(max(1, len(enc_items)), dtype=torch.int32, device=dev)
    lc.check(lc.lc_run_batch(ctx.handle, lc.Batch(enc_items), st_setup, lc.LC_PARALLEL, stream))
    items = []
    for m in range(count):
        if dirs[m] == 0:
            items.append((pws[m], 0, Parena.data_ptr() + p_off[m], int(sizes[m]),
                          Oarena.data_ptr() + o_off[m], clen[m]))
        else:
            items.append((pws[m], 1, Carena.data_ptr() + c_off[m], clen[m],
                          Oarena.data_ptr() + o_off[m], int(sizes[m])))
    batch = lc.Batch(items)
    status = torch.zeros(count, dtype=torch.int32, device=dev)
    msg_bytes = int(sizes.sum())

    # ---- warm-up (also checks every verdict)
    for _ in range(args.warmup):
        lc.check(lc.lc_run_batch(ctx.handle, batch, status, lc.LC_PARALLEL, stream))
    torch.cuda.synchronize()
    bad = int((status != 0).sum())
    if bad:
        raise SystemExit("warm-up: %d requests failed" % bad)
    dec_ok = all(torch.equal(Oarena[o_off[m]:o_off[m] + int(sizes[m])],
                             Parena[p_off[m]:p_off[m] + int(sizes[m])])
                 for m in range(count) if dirs[m] == 1)
    if not dec_ok:
        raise SystemExit("warm-up: a decryption did not reproduce its plaintext")

    # ---- timed region (device-resident inputs)
    lc.check(lc.lc_ctx_timing(ctx.handle, True))
    launches0 = lc.lc_ctx_launch_count(ctx.handle)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        lc.check(lc.lc_run_batch(ctx.handle, batch, status, lc.LC_PARALLEL, stream))
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    elapsed_ms = e0.elapsed_time(e1)
    gpu_launches = lc.lc_ctx_launch_count(ctx.handle) - launches0
    kern_ms, kern_n = lc.lc_ctx_kernel_time(ctx.handle)
    lc.check(lc.lc_ctx_timing(ctx.handle, False))
    elapsed_ms = max_over_ranks(elapsed_ms, dev if ws > 1 else None)
    value = ws * msg_bytes * args.steps / (elapsed_ms * 1e-3) / 1e9
    ms_per_step = elapsed_ms / args.steps

    # ---- roofline of the cipher kernel
    prm = lc.lc_ctx_get_params(ctx.handle)
    ops, parts, traj_bytes = fp64_ops_per_launch(sizes, prm.n_warm, prm.steps_per_byte,
                                                  prm.block_len, prm.tag_len)
    kern_avg_ms = kern_ms / max(1, kern_n)
    achieved = ops / (kern_avg_ms * 1e-3) / 1e9  # G FP64 ops / s
    pipes = lc.lc_probe_pipes(local)
    peak = NOMINAL_FP64_TFLOPS * 1e3 / 2.0
    traffic = committed_traffic(launch.dense_build)
    mask = lc.lc_emu_mask()
    warm_mask = lc.lc_warm_mask()
    hw_ops = fp64_pipe_ops_per_launch(sizes, mask, prm.n_warm, prm.steps_per_byte,
                                      prm.block_len, prm.tag_len, warm_mask)
    hw_rate = hw_ops / (kern_avg_ms * 1e-3) / 1e9
    rl_terms = roofline_terms(sizes, kern_avg_ms, pipes, clk.get("sm_mhz") or pipes.sm_clock_mhz,
                              prm.n_warm, prm.steps_per_byte, prm.block_len, prm.tag_len,
                              launch.dense_build)
    roofline = {
        "bound": "alu", "unit": "G FP64 op/s", "achieved": achieved, "peak": peak,
        "frac": achieved / peak,
        "frac_label": "FP64-only roof, nominal: every binary64 operation of the path against the "
                      "nominal FP64 slot rate",
        "joint": rl_terms["joint"],
        "method_roofline_GBps": rl_terms["method_roofline_GBps"],
        "peak_source": "of fallback: recipe nominal 1.25 TFLOP/s FP64 / 2 flops per DFMA slot "
                       "(no FP64 entry in the measured peaks)",
        "peak_probe": pipes.dadd_gops, "frac_of_probe": achieved / pipes.dadd_gops,
        "ops_per_launch": ops, "kernel_ms": kern_avg_ms, "kernel": "batch_kernel",
        "traffic": traffic["dram_bytes_per_message_byte"] * msg_bytes if traffic else None,
        "traffic_source": ("ncu capture of the same build on one %s, scaled by message bytes"
                           % traffic["captured_case"]) if traffic else None,
        "hbm_bytes_algorithmic": 2 * msg_bytes + 8 * parts,
        "note": "achieved counts every binary64 operation of the path; the kernel runs the "
                "ones in emu_mask as bit-exact integer arithmetic on the INT pipes, so it "
                "exceeds the FP64-pipe peak; fp64_pipe_* is the part that runs on the FP64 pipe",
        "emu_mask": hex(mask), "warm_mask": hex(warm_mask),
        "fp64_pipe_ops_per_launch": hw_ops,
        "fp64_pipe_achieved": hw_rate,
        "fp64_pipe_frac_of_probe": hw_rate / pipes.dadd_gops,
    }

    # ---- per-message launches (same messages, one request per call)
    pm = None
    if args.per_message_sample and rank == 0:
        rng = np.random.default_rng(7)
        order = np.argsort(sizes)
        pick = order[np.linspace(0, count - 1, min(count, args.per_message_sample)).astype(int)]
        s1 = torch.zeros(1, dtype=torch.int32, device=dev)
        singles = [lc.Batch([items[m]]) for m in pick]
        for b in singles[:8]:
            lc.lc_run_batch(ctx.handle, b, s1, lc.LC_PARALLEL, stream)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for b in singles:
            lc.check(lc.lc_run_batch(ctx.handle, b, s1, lc.LC_PARALLEL, stream))
        a1.record(stream)
        torch.cuda.synchronize()
        pm_bytes = int(sizes[pick].sum())
        pm_ms = a0.elapsed_time(a1)
        pm_val = pm_bytes / (pm_ms * 1e-3) / 1e9
        pm = {"value": pm_val, "unit": UNIT, "messages": len(pick),
              "sample": "size-stratified messages of the same workload, one lc_run_batch each",
              "batched_over_per_message": value / ws / pm_val}
        del rng

    # ---- end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        hin_tot = sum(it[3] for it in items)
        hout_tot = sum(it[5] for it in items)
        hin = torch.empty(hin_tot, dtype=torch.uint8).pin_memory()
        # one set of outputs and statuses per batch the library keeps in
        # flight: a step's results stay intact while later steps' copies run
        NS = lc.LC_HOST_INFLIGHT
        houts = [torch.empty(hout_tot, dtype=torch.uint8).pin_memory() for _ in range(NS)]
        hitems = [[] for _ in range(NS)]
        a, b_ = 0, 0
        for m, it in enumerate(items):
            src = Parena if it[1] == 0 else Carena
            off = (p_off[m] if it[1] == 0 else c_off[m])
            hin[a:a + it[3]].copy_(src[off:off + it[3]])
            for j in range(NS):
                hitems[j].append((it[0], it[1], hin.data_ptr() + a, it[3], houts[j].data_ptr() + b_, it[5]))
            a += it[3]
            b_ += it[5]
        hbatches = [lc.Batch(hitems[j]) for j in range(NS)]
        hstats = [np.zeros(count, dtype=np.int32) for _ in range(NS)]
        for j in range(NS):
            lc.check(lc.lc_run_batch_host(ctx.handle, hbatches[j], hstats[j], lc.LC_PARALLEL, stream))
            assert (hstats[j] == 0).all()
        # one synchronous call per step
        barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            lc.check(lc.lc_run_batch_host(ctx.handle, hbatches[k % NS], hstats[k % NS], lc.LC_PARALLEL,
                                          stream))
            if not (hstats[k % NS] == 0).all():
                raise RuntimeError("host-buffer batch failed")
        t_sync = max_over_ranks(time.perf_counter() - t0, dev if ws > 1 else None)
        # pipelined: up to NS - 1 steps are submitted ahead of the one whose
        # results are read, so uploads, kernels and downloads of neighbouring
        # steps overlap
        barrier()
        t0 = time.perf_counter()
        queue = collections.deque()

        def retire():
            t_old, j_old = queue.popleft()
            lc.check(lc.lc_wait_batch_host(ctx.handle, t_old), "lc_wait_batch_host")
            if not (hstats[j_old] == 0).all():
                raise RuntimeError("host-buffer batch failed")
            return j_old

        last = None
        for k in range(args.steps):
            rc, t = lc.lc_submit_batch_host(ctx.handle, hbatches[k % NS], hstats[k % NS], lc.LC_PARALLEL,
                                            stream)
            lc.check(rc, "lc_submit_batch_host")
            queue.append((t, k % NS))
            if len(queue) >= NS:
                last = retire()
        while queue:
            last = retire()
        t_e2e = max_over_ranks(time.perf_counter() - t0, dev if ws > 1 else None)
        e2e = {"value": ws * msg_bytes * args.steps / t_e2e / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": hin_tot, "d2h_bytes_per_step": hout_tot + 4 * count,
               "call": "lc_submit_batch_host + lc_wait_batch_host (%d steps in flight)" % NS,
               "sync_value": ws * msg_bytes * args.steps / t_sync / 1e9,
               "sync_call": "lc_run_batch_host (one synchronous call per step)"}
        # the host path's outputs equal the device path's byte for byte
        # (a sample of messages; outside the timed region)
        rng = np.random.default_rng(11)
        pick = sorted(set(int(x) for x in rng.integers(0, count, 64)) | {0, count - 1})
        b_off, a = [], 0
        for it in items:
            b_off.append(a)
            a += it[5]
        for m in pick:
            n_out = items[m][5]
            got = houts[last][b_off[m]:b_off[m] + n_out]
            want = Oarena[o_off[m]:o_off[m] + n_out].cpu()
            if not torch.equal(got, want):
                raise RuntimeError("host-buffer output of message %d differs from the device path" % m)
        e2e["outputs_checked"] = len(pick)
        del hin, houts, hbatches

    # ---- single-message configurations (64 KiB, 1 MiB both modes, 1 GiB)
    del Parena, Carena, Oarena
    torch.cuda.empty_cache()
    configs = None
    if not args.no_configs:
        configs = single_message_configs(ctx, dev, stream, pipes, clk.get("sm_mhz") or pipes.sm_clock_mhz)

    # ---- served workload (continuous batching), rank 0
    served, served_sample = None, None
    if rank == 0 and args.serve_seconds > 0:
        served, served_sample = run_serving(args.serve_seconds, args.serve_rate, local, value / ws,
                                            args.serve_policy, args.serve_batch_mib,
                                            args.serve_low_seconds, args.serve_capture, args.serve_streams)

    # ---- CPU oracle baseline
    cpu = None
    if rank == 0 and ws == 1 and args.cpu_sample_mb:
        threads = os.cpu_count() or 1
        plan = oracle_sample_plan(spec, args.cpu_sample_mb << 20)
        b_cpu, s_cpu = run_oracle_sample(spec, plan, threads)
        cpu = {"value": b_cpu / s_cpu / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%.0f MiB: the first parts of every message in proportion to its size"
                         % (b_cpu / 2 ** 20),
               "wall_s": s_cpu, "cpu_s_max": s_cpu * threads}
        # the same oracle on one core, on a smaller sample of the same kind
        plan1 = oracle_sample_plan(spec, max(1, args.cpu_sample_mb // 32) << 20)
        b1, s1 = run_oracle_sample(spec, plan1, 1)
        cpu["single_core"] = {"value": b1 / s1 / 1e9, "unit": UNIT, "cores": 1,
                              "sample": "%.0f MiB" % (b1 / 2 ** 20), "wall_s": s1}
        if not args.no_configs:
            cpu["configs"] = oracle_config_rates(threads)
        # the served configuration: the oracle on the captured sample, which
        # also checks every captured ciphertext byte for byte
        if served_sample:
            rec, checked, bad = oracle_check_served(served_sample, threads)
            cpu["served_sample"] = rec
            served[served_sample["label"]]["ciphertext_checked"] = checked
            served[served_sample["label"]]["ciphertext_mismatches"] = bad
            served_sample = None

    if served and pm:
        for rec in served.values():
            rec["served_over_per_message"] = rec["served_GBps"] / pm["value"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 messages and passwords)",
            "config": {"workload": WORKLOAD, "messages": count, "message_bytes": msg_bytes,
                       "parts": parts, "mode": "parallel",
                       "l2": "inputs larger than L2 (%.2f GB per step)" % (msg_bytes / 1e9),
                       "launch": {"threads_per_cta": launch.threads_per_cta,
                                  "ctas_per_sm": launch.ctas_per_sm,
                                  "dense_build": launch.dense_build,
                                  "source": "lc_tune" if tuning else "default"},
                       "tuning": tuning,
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
            "per_message_launch": pm, "served": served, "clocks": clk,
            "configs": configs,
            "pipes_probe_gops": {k: round(v, 1) for k, v in pipes.as_dict().items()},
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
