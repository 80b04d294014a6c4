"""Test helper: the CPU oracle and the seeded input generator on all host
cores.

The oracle's calls are ctypes calls, which release the GIL, so Python
threads run independent parts of a message (Sec. 5: each part is its own
trajectory) at the same time; the output is the oracle's, byte for byte,
whatever the number of threads.  Nothing here computes any of the cipher's
arithmetic itself.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle as O
from paper_1201_3114_gb300 import synth

THREADS = os.cpu_count() or 1
CHUNK_PARTS = 64   # parts per oracle call
GEN_CHUNK = 32 << 20


def uniform(seed, n, offset=0, threads=THREADS):
    """synth.uniform_bytes(seed, n, offset), generated in slices on all cores."""
    out = np.empty(n, dtype=np.uint8)

    def fill(a):
        b = min(n, a + GEN_CHUNK)
        out[a:b] = synth.uniform_bytes(seed, b - a, offset + a)

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(fill, range(0, n, GEN_CHUNK)))
    return out


def uniform_many(seeds, sizes, threads=THREADS):
    """One uniform stream per message (message m: seeds[m], sizes[m] bytes)."""
    outs = [None] * len(seeds)

    def one(m):
        outs[m] = synth.uniform_bytes(seeds[m], int(sizes[m]))

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(one, range(len(seeds))))
    return outs


def encrypt_many(msgs, prm=None, threads=THREADS):
    """Oracle ciphertexts of (password, plaintext) pairs in parallel mode; the
    parts of every message are spread over the threads."""
    prm = prm or O.params()
    B = prm.block_len
    keys = [O.key_schedule(pw, prm) for pw, _ in msgs]
    outs = [np.zeros(O.ciphertext_len(P.size, O.PARALLEL, prm), dtype=np.uint8) for _, P in msgs]
    jobs = []
    for m, (_, P) in enumerate(msgs):
        nb = max(1, -(-P.size // B))
        for b0 in range(0, nb, CHUNK_PARTS):
            jobs.append((m, b0, min(nb, b0 + CHUNK_PARTS)))
    # largest messages first keeps the pool busy to the end
    jobs.sort(key=lambda j: -msgs[j[0]][1].size)

    def run(job):
        m, b0, b1 = job
        P = np.ascontiguousarray(msgs[m][1], dtype=np.uint8)
        O.encrypt_blocks(keys[m], P, P.size, outs[m], b0, b1, prm)

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(run, jobs))
    return outs


def encrypt(pw, P, prm=None, threads=THREADS):
    """Oracle ciphertext of one parallel-mode message on all cores."""
    return encrypt_many([(pw, P)], prm, threads)[0]


def first_difference(a, b):
    """Index of the first differing byte of two equal-length arrays, or -1."""
    if a.size != b.size:
        return min(a.size, b.size)
    d = np.flatnonzero(a != b)
    return int(d[0]) if d.size else -1
