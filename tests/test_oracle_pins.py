"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  None of them compares the oracle
with itself: the expected values are hand derivations (tests/golden/),
closed forms, textbook routines (the Caesar cipher of Sec. 1, hashlib's
SHA-256, a Runge-Kutta integration of the Lorenz system), exact integer
arithmetic, or invariants of the method.
"""
import hashlib
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1201_3114_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line.split("|")


# --------------------------------------------------------------------------
# Eq. 1 (Sec. 3.1): the Euler step of the Lorenz system
# --------------------------------------------------------------------------

def lorenz_field(x, y, z, s=10.0, r=28.0, b=8.0 / 3.0):
    """The Lorenz vector field (textbook form)."""
    return np.array([s * (y - x), r * x - y - x * z, x * y - b * z])


def test_euler_origin_is_fixed(prm):
    assert O.euler_step((0.0, 0.0, 0.0), prm) == (0.0, 0.0, 0.0)


def test_euler_z_axis_invariant(prm):
    # On x = y = 0 the field is (0, 0, -beta z): x, y stay exactly 0 and z
    # decays geometrically by (1 - beta dt) per step up to rounding.
    r = (0.0, 0.0, 25.0)
    for n in range(1, 200):
        r = O.euler_step(r, prm)
        assert r[0] == 0.0 and r[1] == 0.0
        expect = 25.0 * (1.0 - (8.0 / 3.0) * 0.01) ** n
        assert abs(r[2] - expect) <= 1e-12 * 25.0


def test_euler_nontrivial_fixed_points(prm):
    # C+- = (+-sqrt(beta(rho-1)), +-sqrt(beta(rho-1)), rho-1): the field vanishes,
    # so one step moves by a few rounding errors only.
    c = math.sqrt((8.0 / 3.0) * 27.0)
    for sgn in (1.0, -1.0):
        r0 = (sgn * c, sgn * c, 27.0)
        r1 = O.euler_step(r0, prm)
        assert max(abs(a - b) for a, b in zip(r0, r1)) < 1e-13


def test_euler_matches_lorenz_field(prm):
    # (F(r) - r) / dt must equal the Lorenz field: catches a dropped term,
    # a wrong sign or a swapped operand in any component.
    rng = np.random.default_rng(7)
    for _ in range(200):
        r = rng.uniform([-20, -25, 0], [20, 25, 50])
        f = lorenz_field(*r)
        got = (np.array(O.euler_step(tuple(r), prm)) - r) / prm.dt
        assert np.allclose(got, f, rtol=1e-9, atol=1e-9), (r, got, f)


def _rk4(r, h, n):
    r = np.array(r, dtype=np.float64)
    for _ in range(n):
        k1 = lorenz_field(*r)
        k2 = lorenz_field(*(r + 0.5 * h * k1))
        k3 = lorenz_field(*(r + 0.5 * h * k2))
        k4 = lorenz_field(*(r + h * k3))
        r = r + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return r


def test_euler_first_order_convergence():
    # Forward Euler is first order: over t in [0, 0.5] from (1, 1, 20) the
    # error against a fine RK4 solution halves as dt halves.
    T = 0.5
    ref = _rk4((1.0, 1.0, 20.0), 1e-4, int(round(T / 1e-4)))
    errs = []
    for dt in (0.01, 0.005, 0.0025, 0.00125):
        p = O.params(dt=dt)
        r = (1.0, 1.0, 20.0)
        for _ in range(int(round(T / dt))):
            r = O.euler_step(r, p)
        errs.append(np.linalg.norm(np.array(r) - ref))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    for q in ratios:
        assert 1.8 <= q <= 2.2, (errs, ratios)


# --------------------------------------------------------------------------
# Sec. 3.1 key schedule: Eqs. 2-4, g(x), mu, Eq. 7
# --------------------------------------------------------------------------

@pytest.mark.parametrize("row", list(_rows("key_schedule_worked.txt")), ids=lambda r: r[0])
def test_key_schedule_worked_examples(row, prm):
    pw, a1, a2, a3, L, D, mu = row
    k = O.key_schedule(pw, prm)
    assert k.a == (int(a1), int(a2), int(a3))
    assert (k.L, k.D) == (int(L), int(D))
    if mu != "-":
        assert list(k.mu) == [int(v) for v in mu.split()]


def test_decimal_exponent_table(prm):
    # D = ceil(log10 2^(8(L+1))), L = 0..10, from the closed form.
    for L in range(11):
        pw = b"\x01" * (3 * L + (1 if L == 0 else 0))
        k = O.key_schedule(pw, prm)
        assert k.L == L
        assert k.D == math.ceil(8 * (L + 1) * math.log10(2.0))


def test_aprime_mu_omega_exact(prm):
    # a'_j = RN(RN(a_j) / RN(10^D)) with Python's correctly rounded int->float;
    # mu from unreduced big-integer products; Omega from hashlib (reading R12).
    for length in range(1, 33):
        for rep in range(4):
            pw = synth.password(synth.subseed(99, 100 * length + rep), length)
            k = O.key_schedule(pw, prm)
            a = k.a
            assert all(0 <= v < 2 ** (8 * (k.L + 1)) for v in a)
            for j in range(3):
                assert k.aprime[j] == float(a[j]) / float(10 ** k.D)
                assert 0.0 <= k.aprime[j] < 1.0
            assert k.mu[0] == (a[0] + a[1] + a[2]) % 3
            assert k.mu[1] == (a[0] * a[1] + a[2]) % 3
            assert k.mu[2] == (a[0] + a[1] * a[2]) % 3
            for i in range(3):
                msg = b"".join(((i + 1) * v).to_bytes(16, "little") for v in a)
                h = int.from_bytes(hashlib.sha256(msg).digest(), "big")
                assert k.omega[i] == h % prm.k[i]


def test_key_packing_uses_every_password_byte(prm):
    # Eqs. 2-4 place each of the 3L (+ n mod 3) bytes exactly once: changing
    # any single byte changes a, and the a_i together hold exactly the bytes.
    for length in range(1, 33):
        pw = bytes(range(1, length + 1))
        base = O.key_schedule(pw, prm).a
        total_bits = sum(v.bit_length() > 0 for v in base)
        assert total_bits >= 1
        digits = []
        for v in base:
            while v:
                digits.append(v & 255)
                v >>= 8
        assert sorted(d for d in digits if d) == sorted(pw)
        for i in range(length):
            mod = bytearray(pw)
            mod[i] ^= 0x40
            assert O.key_schedule(bytes(mod), prm).a != base


def test_password_length_limits(prm):
    with pytest.raises(ValueError):
        O.key_schedule(b"", prm)
    with pytest.raises(ValueError):
        O.key_schedule(b"x" * 33, prm)
    O.key_schedule(b"x" * 32, prm)


def test_sha256_matches_hashlib():
    rng = np.random.default_rng(3)
    for n in list(range(0, 130)) + [1000, 4097]:
        m = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        assert O.sha256(m) == hashlib.sha256(m).digest()


# --------------------------------------------------------------------------
# Eq. 8 (R_nu) and Eqs. 9-10 (byte map)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("row", list(_rows("rbyte_worked.txt")), ids=lambda r: r[0])
def test_rbyte_worked_examples(row):
    alpha = float(row[0])
    want = [int(v) for v in row[1].split()]
    assert [O.rbyte(alpha, w) for w in range(4)] == want


def test_rbyte_exact_integer_semantics():
    # floor(RN(alpha 1e13)) in exact integer arithmetic, two's complement bytes.
    rng = np.random.default_rng(11)
    alphas = np.concatenate([rng.uniform(-60, 60, 3000), rng.uniform(-1e-9, 1e-9, 200),
                             [0.0, -0.0, 2.0 ** -60, -(2.0 ** -60), 921.0, -921.0]])
    for a in alphas:
        v = float(a) * 1e13
        V = math.floor(v) % (1 << 64)
        for w in range(8):
            assert O.rbyte(float(a), w) == (V >> (8 * w)) & 255


def test_sat_floor_special_values():
    assert O.sat_floor(float("nan")) == 0
    assert O.sat_floor(float("inf")) == 2 ** 63 - 1
    assert O.sat_floor(float("-inf")) == -(2 ** 63)
    assert O.sat_floor(2.0 ** 63) == 2 ** 63 - 1
    assert O.sat_floor(-(2.0 ** 63)) == -(2 ** 63)
    assert O.sat_floor(-2.5) == -3 and O.sat_floor(2.5) == 2 and O.sat_floor(-0.0) == 0


def test_byte_map_is_caesar_and_invertible():
    # Sec. 1: with R1 + R2 frozen to pi, Eq. 9 is the Caesar cipher
    # (P + pi) mod 2^8 and Eq. 10 is its inverse (the sign flip of the mod).
    for r2 in (0, 1, 128, 255):
        for r1 in range(256):
            pi = r1 + r2
            for x in range(0, 256, 1 if r1 % 17 == 0 else 37):
                y = O.encode_byte(x, r1, r2)
                assert y == (x + pi) % 256
                assert O.decode_byte(y, r1, r2) == x
                assert O.decode_byte(x, r1, r2) == (x - pi) % 256


def _byte_map_slice(r2):
    """Every (x, R1) for one R2: mismatches against the Caesar cipher and
    against D(E(x)) = x (worker of the exhaustive test)."""
    import oracle as Ow
    lib = Ow.lib()
    enc, dec = lib.lco_encode_byte, lib.lco_decode_byte
    bad = 0
    for r1 in range(256):
        pi = r1 + r2
        for x in range(256):
            y = enc(x, r1, r2)
            if y != (x + pi) % 256 or dec(y, r1, r2) != x or dec(x, r1, r2) != (x - pi) % 256:
                bad += 1
    return bad


def test_byte_map_exhaustive():
    # Eqs. 9-10 over all 256^3 (x, R1, R2): the Caesar cipher of Sec. 1 with
    # key R1 + R2, and decryption inverts encryption (the reversibility of
    # the mod stated in Sec. 3.2).  16.7 million cases on a spawn pool.
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, os.cpu_count() or 1)) as pool:
        assert sum(pool.map(_byte_map_slice, range(256), chunksize=8)) == 0


# --------------------------------------------------------------------------
# Sec. 3.2 Steps 1-3 in special cases with frozen dynamics
# --------------------------------------------------------------------------

FROZEN = dict(sigma=0.0, rho=0.0, beta=0.0, dt=0.0)
V15 = 15_000_000_000_000  # floor(1.5 * 10^13), exact
B15 = [(V15 >> (8 * w)) & 255 for w in range(4)]  # (0, 240, 171, 117)


def _nul_key(prm):
    # A password of NUL bytes gives a = 0, a' = 0, mu = (0, 0, 0); every
    # Omega_i hashes the same 48 zero bytes.
    k = O.key_schedule(b"\x00\x00\x00", prm)
    assert k.a == (0, 0, 0) and list(k.mu) == [0, 0, 0]
    h = int.from_bytes(hashlib.sha256(bytes(48)).digest(), "big")
    assert list(k.omega) == [h % 4] * 3
    return k


def test_frozen_dynamics_zero_plaintext_is_caesar():
    # sigma = rho = beta = dt = 0 makes F the identity; with r_0 = (1.5, 1.5, 1.5)
    # and P = 0 the kick is 0, so alpha stays 1.5 and every R is a byte of
    # 15e12 = 0x0DA475ABF000.  Omega then follows the integer map
    # w -> (w + byte_w) mod 4, and the key stream is the Caesar key
    # (R1 + R2) mod 256 of Sec. 1 at each step.
    prm = O.params(lam=(1.5, 1.5, 1.5), n_warm=7, **FROZEN)
    k = _nul_key(prm)
    w = k.omega[0]
    n = 40
    ct = O.encrypt(b"\x00\x00\x00", np.zeros(n, np.uint8), O.SEQUENTIAL, prm)
    want = []
    for _ in range(n):
        want.append((B15[w] + B15[w]) % 256)
        w = (w + B15[w]) % 4
    assert list(ct[:n]) == want


def test_frozen_dynamics_two_byte_trace():
    # One kick in the frozen system.  Byte 0 (P0) is Caesar-coded with the
    # bytes of 1.5e13; Step 2 adds Theta = P0 / 10^(3 + Omega_3) to r[mu_3] = x;
    # Step 3 leaves mu at 0 because every byte of 1.5e13 is 0 mod 3, re-reads
    # alpha = x, and moves Omega with the bytes of floor(x * 1e13).  Byte 1 is
    # coded with those bytes.
    prm = O.params(lam=(1.5, 2.5, 3.5), n_warm=3, **FROZEN)
    k = _nul_key(prm)
    w0 = k.omega[0]
    assert all(b % 3 == 0 for b in B15)
    for p0 in (1, 77, 200, 255):
        for p1 in (0, 9):
            ct = O.encrypt(b"\x00\x00\x00", np.array([p0, p1], np.uint8), O.SEQUENTIAL, prm)
            assert ct[0] == (p0 + 2 * B15[w0]) % 256
            x1 = 1.5 + p0 / 10.0 ** (3 + w0)  # kick into x, identity F, a' = 0
            V = math.floor(x1 * 1e13)
            bx = [(V >> (8 * w)) & 255 for w in range(4)]
            w1 = (w0 + bx[w0]) % 4
            assert ct[1] == (p1 + 2 * bx[w1]) % 256


def test_step3_order_statistic():
    # Reading of Step 3: Omega moves with the new alpha and the old Omega, and
    # the next Step 1 reads the same alpha at the new Omega.  Whenever Omega
    # stays (prob. 1/4) the next R1 is therefore 0 mod 4, so
    # P(R1 = 0 mod 4) = 1/4 + 3/4 * 1/4 = 7/16 exactly; with the old alpha in
    # the Omega update it would be 1/4.
    prm = O.params()
    key = O.key_schedule("123456", prm)
    n = 1 << 19
    P = synth.uniform_bytes(1, n)
    Cb = np.zeros(O.ciphertext_len(n, prm=prm), np.uint8)
    st = O.Stats()
    O.encrypt_blocks(key, P, n, Cb, 0, O.nblocks(n, prm=prm), prm, st)
    h = np.array(st.r1_hist[:], dtype=np.float64)
    share = h[::4].sum() / h.sum()
    assert abs(share - 7.0 / 16.0) < 0.004, share


# --------------------------------------------------------------------------
# The chaos gate: bounded trajectory, uniform low-order digits (Fig. 1 c, d)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("pw", ["123456", "x" * 32, "Qw3rty!Zx9#pL0vB7nM2kT5a"])
def test_chaos_gate(pw):
    import scipy.stats as ss
    prm = O.params()
    key = O.key_schedule(pw, prm)
    n = 1 << 19
    P = synth.uniform_bytes(2, n)
    Cb = np.zeros(O.ciphertext_len(n, prm=prm), np.uint8)
    st = O.Stats()
    O.encrypt_blocks(key, P, n, Cb, 0, O.nblocks(n, prm=prm), prm, st)
    assert st.max_abs_r < 1e3
    h = np.array(st.r1_hist[:], dtype=np.float64)
    # within each residue class mod 4 the low-order byte is uniform
    for res in range(4):
        assert ss.chisquare(h[res::4]).pvalue > 1e-4
    # the ciphertext of uniform data is uniform (Sec. 4, Fig. 2)
    cnt = np.bincount(Cb[:n], minlength=256)
    assert ss.chisquare(cnt).pvalue > 1e-4


# --------------------------------------------------------------------------
# Whole messages: D(E(P)) = P, tamper detection, the parallel split
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [O.PARALLEL, O.SEQUENTIAL])
def test_round_trip(mode):
    prm = O.params()
    B = prm.block_len
    sizes = [0, 1, 15, 16, 17, B - 1, B, B + 1, 2 * B + 7, 3 * B + 5]
    for i, n in enumerate(sizes):
        pw = synth.password(synth.subseed(5, i), 1 + (7 * i) % 32)
        P = synth.uniform_bytes(synth.subseed(6, i), n)
        ct = O.encrypt(pw, P, mode, prm)
        assert ct.size == O.ciphertext_len(n, mode, prm)
        assert O.plaintext_len(ct.size, mode, prm) == n
        st, back = O.decrypt(pw, ct, mode, prm)
        assert st == O.OK and np.array_equal(back, P)
        if n:
            assert not np.array_equal(ct[:n], P)


def test_round_trip_every_password_length():
    prm = O.params()
    P = synth.uniform_bytes(8, 300)
    for length in range(1, 33):
        pw = synth.password(synth.subseed(9, length), length)
        ct = O.encrypt(pw, P, O.PARALLEL, prm)
        assert O.decrypt(pw, ct, O.PARALLEL, prm)[1].tobytes() == P.tobytes()


def test_lengths():
    prm = O.params()
    B, T = prm.block_len, prm.tag_len
    for n in [0, 1, B - 1, B, B + 1, 5 * B, 5 * B + 3]:
        nb = max(1, -(-n // B))
        assert O.ciphertext_len(n, O.PARALLEL, prm) == n + T * nb
        assert O.ciphertext_len(n, O.SEQUENTIAL, prm) == n + T
    valid = {O.ciphertext_len(n, O.PARALLEL, prm) for n in range(0, 3 * B + 50)}
    for c in range(0, 3 * (B + T) + 40):
        got = O.plaintext_len(c, O.PARALLEL, prm)
        assert (got is not None) == (c in valid)
    assert O.plaintext_len(T - 1, O.SEQUENTIAL, prm) is None


def test_tag_flip_always_rejected():
    # A flipped tag byte changes the decoded tag byte through a bijection at a
    # fixed state, so it can never decode to the expected length byte.
    prm = O.params()
    pw = "tamper-test-pw"
    P = synth.uniform_bytes(10, 2 * prm.block_len + 100)
    ct = O.encrypt(pw, P, O.PARALLEL, prm)
    n = P.size
    for pos in range(n, ct.size):
        for bit in (0x01, 0x80):
            bad = ct.copy()
            bad[pos] ^= bit
            st, out = O.decrypt(pw, bad, O.PARALLEL, prm)
            assert st == O.ERR_INTEGRITY and not out.any()


def test_body_flip_rejected():
    # Sec. 2: a change in C_i changes P_i, Theta and the whole later path, so
    # the tag of that part decodes to noise (miss probability 2^-64 each).
    prm = O.params()
    pw = "body-flip"
    P = synth.uniform_bytes(12, 300)
    ct = O.encrypt(pw, P, O.PARALLEL, prm)
    rng = np.random.default_rng(13)
    for _ in range(2000):
        bad = ct.copy()
        pos = int(rng.integers(0, P.size))
        bad[pos] ^= int(rng.integers(1, 256))
        assert O.decrypt(pw, bad, O.PARALLEL, prm)[0] == O.ERR_INTEGRITY


def test_wrong_password_rejected():
    prm = O.params()
    P = synth.uniform_bytes(14, 5000)
    ct = O.encrypt("123456", P, O.PARALLEL, prm)
    st, out = O.decrypt("123457", ct, O.PARALLEL, prm)
    assert st == O.ERR_INTEGRITY and not out.any()


def test_parallel_equals_sequential_for_one_part():
    # Sec. 5: with a single part the parallel split is the sequential method.
    prm = O.params()
    for n in (0, 1, 100, prm.block_len):
        P = synth.uniform_bytes(15, n)
        assert np.array_equal(O.encrypt("pw-seq-par", P, O.PARALLEL, prm),
                              O.encrypt("pw-seq-par", P, O.SEQUENTIAL, prm))


def test_parallel_is_per_part_sequential():
    # Sec. 5: each part is an independent trajectory started at its own
    # initial condition; its tag follows the body of that part.
    prm = O.params(block_len=64, n_warm=50)
    pw = "split"
    key = O.key_schedule(pw, prm)
    n = 64 * 3 + 10
    P = synth.uniform_bytes(16, n)
    ct = O.encrypt(pw, P, O.PARALLEL, prm)
    Q = list(n.to_bytes(8, "little"))
    for b in range(4):
        st = O.block_begin(key, b, prm)
        body = [O.step_byte(key, st, int(x), O.ENCRYPT, prm) for x in P[64 * b:64 * (b + 1)]]
        tag = [O.step_byte(key, st, q, O.ENCRYPT, prm) for q in Q]
        assert body == list(ct[64 * b:64 * b + len(body)])
        assert tag == list(ct[n + 8 * b:n + 8 * b + 8])
    # parts start from distinct points (r_0 + b eta)
    s0, s1 = O.block_begin(key, 0, O.params(block_len=64, n_warm=0)), \
        O.block_begin(key, 1, O.params(block_len=64, n_warm=0))
    assert all(b - a == 2.0 ** -24 for a, b in zip(s0.r, s1.r))


def test_password_sensitivity():
    # Sec. 4, Fig. 2: "123456" and "123457" give unrelated ciphertexts.
    prm = O.params()
    P = synth.zipf_text(17, 1 << 16)
    c1 = O.encrypt("123456", P, O.PARALLEL, prm)
    c2 = O.encrypt("123457", P, O.PARALLEL, prm)
    assert np.mean(c1 != c2) >= 0.99


def test_ciphertext_entropy():
    # Sec. 4: the ciphertext entropy reaches the 8-bit maximum.
    prm = O.params()
    P = synth.uniform_bytes(18, 1 << 20)
    c = O.encrypt("entropy-check", P, O.PARALLEL, prm)[:P.size]
    p = np.bincount(c, minlength=256) / c.size
    H = -(p[p > 0] * np.log2(p[p > 0])).sum()
    assert H >= 7.99


def test_zero_run_does_not_repeat():
    # Sec. 2: repeated plaintext must not give repeated ciphertext: no short
    # period and adjacent repeats at the rate of a random sequence.
    prm = O.params()
    c = O.encrypt("zeros", np.zeros(4096, np.uint8), O.PARALLEL, prm)[:4096].astype(int)
    assert np.sum(c[1:] == c[:-1]) < 100
    for period in range(1, 257):
        assert np.mean(c[period:] == c[:-period]) < 0.1


def test_step3_symmetric_lock_is_absorbing():
    # Step 3 applies the same rule to every i (and k_1 = k_2 = k_3), so once
    # (mu_i, Omega_i) = (mu_j, Omega_j) the two stay equal for good: then
    # alpha_i = alpha_j, R1 = R2 and C - P = 2 R1 is even.
    prm = O.params()
    key = O.key_schedule("123456", prm)
    st = O.block_begin(key, 0, prm)
    P = synth.uniform_bytes(20, 4096)
    locked = set()
    for x in P:
        before = st.copy()
        y = O.step_byte(key, st, int(x), O.ENCRYPT, prm)
        r1 = O.rbyte(before.alpha[0], before.omega[0])
        r2 = O.rbyte(before.alpha[1], before.omega[1])
        assert y == (int(x) + r1 + r2) % 256
        for i, j in ((0, 1), (0, 2), (1, 2)):
            same = before.mu[i] == before.mu[j] and before.omega[i] == before.omega[j]
            if (i, j) in locked:
                assert same
            if same:
                locked.add((i, j))
                assert before.alpha[i] == before.alpha[j]
                assert st.mu[i] == st.mu[j] and st.omega[i] == st.omega[j]
    assert (0, 1) in locked
    c = O.encrypt("123456", P, O.PARALLEL, prm)[:4096].astype(int)
    assert np.all((c[64:] - P[64:].astype(int)) % 2 == 0)


def test_divergent_profile_is_deterministic():
    # dt = 0.027 (the top of the paper's range) with the +a' forcing leaves the
    # basin and reaches non-finite values; NaN bytes saturate to 0 and the
    # round trip still holds.
    prm = O.params(dt=0.027)
    P = synth.uniform_bytes(19, 9000)
    c = O.encrypt("123456", P, O.PARALLEL, prm)
    assert np.array_equal(O.decrypt("123456", c, O.PARALLEL, prm)[1], P)
