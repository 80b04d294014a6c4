"""Seeded synthetic inputs: the only module shared by the CUDA path's tests
and the oracle's.  It holds none of the cipher's arithmetic.

Every random draw comes from SplitMix64 (Steele, Lea & Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) used as a
counter-based generator: word i of stream ``seed`` is
``mix(seed + (i + 1) * GAMMA)``, byte j of a uniform byte stream is byte
``j mod 8`` (little-endian) of word ``j // 8``.  The CUDA library carries its
own device implementation of the same published definition
(``lc_synth_uniform``) so that gigabyte inputs can be made on the device;
the two are cross-checked by a test.

Workload recipes (sizes and distributions of the paper's experiments, which
used a book and an image that are not available here):
  * uniform random bytes (Sec. 4 image / generic binary data),
  * text-like bytes: Zipf s=1.1 over the 95 printable ASCII codes, rank r
    mapped to code 31 + r so the space is the most frequent symbol, with a
    4 KiB all-zero run at a seeded offset (stand-in for the book of Sec. 4),
  * passwords of printable ASCII, char = 32 + (u mod 95),
  * log-uniform message sizes for batched and served runs.
"""
import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
MASK64 = (1 << 64) - 1

CONFIG_SEED_BASE = 0x1201_3114_0000


def config_seed(c: int) -> int:
    """Seed of workload configuration c (1..5)."""
    return CONFIG_SEED_BASE + c


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def words(seed: int, start: int, count: int) -> np.ndarray:
    """Words start .. start+count-1 of stream ``seed`` (uint64)."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + idx * GAMMA
    return _mix(z)


def word(seed: int, i: int) -> int:
    return int(words(seed, i, 1)[0])


def subseed(seed: int, label: int) -> int:
    """An independent stream derived from ``seed`` for purpose ``label``."""
    return word(seed ^ 0x5DEECE66D, label)


def uniform_bytes(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Bytes offset .. offset+n-1 of the uniform byte stream ``seed``."""
    if n <= 0:
        return np.zeros(0, dtype=np.uint8)
    w0 = offset // 8
    w1 = (offset + n + 7) // 8
    raw = words(seed, w0, w1 - w0).astype("<u8").view(np.uint8)
    s = offset - 8 * w0
    return raw[s:s + n].copy()


def unit_doubles(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each word."""
    return (words(seed, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def password(seed: int, length: int) -> bytes:
    """``length`` printable ASCII characters (codes 32..126)."""
    w = words(seed, 0, length)
    return bytes(int(32 + (int(x) % 95)) for x in w)


def passwords_bulk(seeds: np.ndarray, lo: int = 8, hi: int = 32):
    """Vectorised ``password(s, password_len(s, lo, hi))`` for many seeds:
    (uint8 array [len(seeds), hi] zero-padded, int64 lengths)."""
    seeds = np.asarray(seeds, dtype=np.uint64)
    n = seeds.size
    with np.errstate(over="ignore"):
        lw = _mix(seeds + np.uint64(1_000_003 + 1) * GAMMA)
        lengths = (lo + (lw % np.uint64(hi - lo + 1)).astype(np.int64))
        j = np.arange(1, hi + 1, dtype=np.uint64)
        z = seeds[:, None] + j[None, :] * GAMMA
        chars = (32 + (_mix(z) % np.uint64(95))).astype(np.uint8)
    mask = np.arange(hi)[None, :] < lengths[:, None]
    chars[~mask] = 0
    return chars, lengths


def password_len(seed: int, lo: int, hi: int) -> int:
    """A length uniform in [lo, hi]."""
    return lo + word(seed, 1_000_003) % (hi - lo + 1)


def zipf_text(seed: int, n: int, s: float = 1.1, zero_run: int = 4096) -> np.ndarray:
    """Text-like bytes: Zipf(s) over ranks 1..95 mapped to codes 31 + rank,
    then ``zero_run`` zero bytes written at a seeded offset in [0, n - zero_run]."""
    ranks = np.arange(1, 96, dtype=np.float64)
    pmf = ranks ** (-s)
    cdf = np.cumsum(pmf / pmf.sum())
    cdf[-1] = 1.0
    u = unit_doubles(seed, 0, n)
    r = np.searchsorted(cdf, u, side="right") + 1  # rank 1..95
    out = (31 + r).astype(np.uint8)
    if zero_run and n >= zero_run:
        off = word(seed, n + 17) % (n - zero_run + 1)
        out[off:off + zero_run] = 0
    return out


def log_uniform_sizes(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """floor(exp(U(ln lo, ln hi))) for ``count`` draws (int64)."""
    u = unit_doubles(seed, 0, count)
    v = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))))
    return np.clip(v, lo, hi).astype(np.int64)


# --------------------------------------------------------------------------
# The five workload configurations
# --------------------------------------------------------------------------

def cfg1():
    """64 KiB uniform bytes, 16-char password, parallel mode."""
    sd = config_seed(1)
    return dict(pw=password(subseed(sd, 1), 16), P=uniform_bytes(subseed(sd, 2), 65536))


def cfg2():
    """1 MiB Zipf text with a 4 KiB zero run, 32-char password, both modes;
    the seeded ciphertext offset to flip for the integrity test."""
    sd = config_seed(2)
    n = 1 << 20
    return dict(pw=password(subseed(sd, 1), 32), P=zipf_text(subseed(sd, 2), n),
                flip_seed=subseed(sd, 3))


def cfg3_spec():
    """1 GiB uniform bytes (made on the device from ``data_seed``), 24-char password."""
    sd = config_seed(3)
    return dict(pw=password(subseed(sd, 1), 24), data_seed=subseed(sd, 2), n=1 << 30)


def cfg4_spec(count: int = 4096, lo: int = 1024, hi: int = 4 << 20):
    """Batched workload: ``count`` messages, log-uniform sizes in [lo, hi],
    8-32-char passwords, the first half encrypted and the second half
    decrypted.  Message m's plaintext is the uniform stream ``data_seed(m)``."""
    sd = config_seed(4)
    sizes = log_uniform_sizes(subseed(sd, 1), count, lo, hi)
    pws = []
    for m in range(count):
        ps = subseed(sd, 1000 + m)
        pws.append(password(ps, password_len(ps, 8, 32)))
    data_seeds = [subseed(sd, 100000 + m) for m in range(count)]
    dirs = [0 if m < count // 2 else 1 for m in range(count)]
    return dict(sizes=sizes, pws=pws, data_seeds=data_seeds, dirs=dirs)


def cfg5_spec(rate: float = 20000.0, duration: float = 60.0, lo: int = 256,
              hi: int = 16 << 20, tamper_frac: float = 0.02):
    """Served workload: Poisson arrivals (exponential gaps), log-uniform sizes,
    50/50 encrypt/decrypt, 8-32-char passwords, a fraction of decrypts with one
    tampered byte.  Returns numpy arrays describing every request."""
    sd = config_seed(5)
    expect = int(rate * duration * 1.2) + 64
    gaps = -np.log1p(-unit_doubles(subseed(sd, 1), 0, expect)) / rate
    t = np.cumsum(gaps)
    count = int(np.searchsorted(t, duration, side="left"))
    t = t[:count]
    sizes = log_uniform_sizes(subseed(sd, 2), count, lo, hi)
    kind = (words(subseed(sd, 3), 0, count) & np.uint64(1)).astype(np.int8)  # 1 = decrypt
    tam = unit_doubles(subseed(sd, 4), 0, count) < tamper_frac
    tamper = (kind == 1) & tam
    pw_seed = words(subseed(sd, 5), 0, count)
    data_seed = words(subseed(sd, 6), 0, count)
    flip_pos = words(subseed(sd, 7), 0, count)
    return dict(t=t, sizes=sizes, kind=kind, tamper=tamper, pw_seed=pw_seed,
                data_seed=data_seed, flip_pos=flip_pos)
