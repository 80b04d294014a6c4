"""Closed-form pins of the oracle's per-byte recurrence (Sec. 3.2, Steps 1-3),
of the trajectory start (Eq. 5 plus the part offset of Sec. 5, Eq. 6 for
alpha) and of the warm-up length (n_it, Sec. 3.1).

The oracle exposes its per-trajectory state, so each test sets r, alpha, mu
and Omega by hand, runs one byte (or one trajectory start) and compares the
new state with values that follow from the paper's equations in special
cases where one Euler step of the Lorenz system (Eq. 1) has a closed form:

  * on the z-axis (x = y = 0) the field is (0, 0, -beta z): x and y stay
    exactly 0 and one step multiplies z by (1 - beta dt);
  * at (0, y, z) the field is (sigma y, -y, -beta z), so one step gives
    (dt sigma y, (1 - dt) y, (1 - beta dt) z).

Step 2 of Sec. 3.2 kicks the component r[mu_3] by Theta = P / 10^(3 + Omega_3)
and then applies F (r_i = F[r_{i-1} + M(P_i)], Sec. 2); Step 3 moves mu with
the old alpha and Omega, re-reads alpha from r with the new mu (Eq. 6), moves
Omega with the new alpha and the old Omega, and adds a' to r last (the order
of reading R13).  R_nu (Eq. 8) is computed here with exact integer
arithmetic (pinned on its own in test_oracle_pins.py).  Each test first
checks that the plausible misreadings it guards against would predict a
different result, so a pass is not an accident of the chosen values.
"""
import math

import numpy as np
import pytest

import oracle as O

BETA = 8.0 / 3.0


def rb(alpha, omega):
    """R_nu(alpha, Omega) of Eq. 8, nu = 13, from the exact integer floor."""
    v = math.floor(alpha * 1e13) % (1 << 64)
    return (v >> (8 * omega)) & 255


def key(aprime=(0.0, 0.0, 0.0), mu=(0, 0, 0), omega=(0, 0, 0)):
    k = O.Key()
    for j in range(3):
        k.aprime[j] = aprime[j]
        k.mu[j] = mu[j]
        k.omega[j] = omega[j]
    return k


def state(r, alpha, mu, omega):
    s = O.State()
    for j in range(3):
        s.r[j] = r[j]
        s.alpha[j] = alpha[j]
        s.mu[j] = mu[j]
        s.omega[j] = omega[j]
    return s


def close(a, b, rel=1e-13):
    return abs(a - b) <= rel * max(abs(a), abs(b), 1e-300)


# --------------------------------------------------------------------------
# Step 2: the kick lands on r[mu_3], Theta = P / 10^(3 + Omega_3), then F
# --------------------------------------------------------------------------

@pytest.mark.parametrize("direction", [O.ENCRYPT, O.DECRYPT])
def test_step2_kick_on_z_axis_then_one_euler_step(prm, direction):
    # mu = (0, 1, 2): the kick goes to z and x = y = 0 survives the step
    # exactly.  Kick then F gives z' = (z0 + Theta)(1 - beta dt); F then kick
    # would give z0 (1 - beta dt) + Theta; a kick on r[mu_1] = x would leave
    # x != 0.
    dt = prm.dt
    z0 = 20.0
    alpha = (1.5, -1.5, 2.5)
    for w3 in range(4):
        for x in (0, 1, 77, 200, 255):
            st = state((0.0, 0.0, z0), alpha, (0, 1, 2), (1, 2, w3))
            y = O.step_byte(key(), st, x, direction, prm)
            s = rb(alpha[0], 1) + rb(alpha[1], 2)
            P = x if direction == O.ENCRYPT else (x - s) % 256
            assert y == ((x + s) % 256 if direction == O.ENCRYPT else P)
            theta = P / 10.0 ** (3 + w3)
            want = (z0 + theta) * (1.0 - BETA * dt)
            if P:
                assert not close(want, z0 * (1.0 - BETA * dt) + theta, 1e-9)
                # Theta with Omega_1 (= 1) or without the 10^3 would differ
                assert not close(want, (z0 + P / 10.0 ** 4) * (1.0 - BETA * dt), 1e-9) or w3 == 1
            assert st.r[0] == 0.0 and st.r[1] == 0.0, (w3, x)
            assert close(st.r[2], want), (w3, x, st.r[2], want)


def test_step2_kick_on_y_then_one_euler_step(prm):
    # mu_3 = 1: r = (0, 0, z0) becomes (0, Theta, z0) and one Euler step
    # gives (dt sigma Theta, (1 - dt) Theta, (1 - beta dt) z0).  F before the
    # kick would leave x = 0; a kick on mu_1 = 2 would leave y = 0.
    dt = prm.dt
    z0 = 30.0
    for w3, x in ((0, 255), (1, 9), (2, 128), (3, 1)):
        st = state((0.0, 0.0, z0), (0.25, 0.5, 0.75), (2, 0, 1), (0, 0, w3))
        O.step_byte(key(), st, x, O.ENCRYPT, prm)
        th = x / 10.0 ** (3 + w3)
        assert close(st.r[0], dt * 10.0 * th), (w3, x, st.r[0])
        assert close(st.r[1], (1.0 - dt) * th), (w3, x, st.r[1])
        assert close(st.r[2], (1.0 - BETA * dt) * z0), (w3, x, st.r[2])


def test_steps_per_byte_applies_f_s_times(prm):
    # With S applications of F per byte the kicked z-axis state decays by
    # (1 - beta dt)^S.
    for S in (1, 2, 5):
        p = O.params(steps_per_byte=S)
        st = state((0.0, 0.0, 10.0), (1.0, 1.0, 1.0), (0, 1, 2), (0, 0, 0))
        O.step_byte(key(), st, 100, O.ENCRYPT, p)
        assert st.r[0] == 0.0 and st.r[1] == 0.0
        assert close(st.r[2], (10.0 + 0.1) * (1.0 - BETA * p.dt) ** S, 1e-12), S


# --------------------------------------------------------------------------
# Step 3: mu, alpha, Omega and r += a'
# --------------------------------------------------------------------------

def _step3_cases(prm, count):
    """Seeded states (alpha, mu, Omega) on the z-axis for which every
    misreading below predicts a different new state than the reading."""
    rng = np.random.default_rng(2024)
    dt = prm.dt
    out = []
    while len(out) < count:
        alpha = tuple(float(v) for v in rng.uniform(-40.0, 40.0, 3))
        mu = (int(rng.integers(0, 3)), int(rng.integers(0, 3)), 2)  # the kick goes to z
        om = tuple(int(v) for v in rng.integers(0, 4, 3))
        x = int(rng.integers(0, 256))
        z0 = float(rng.uniform(5.0, 45.0))
        ap = tuple(float(v) for v in rng.uniform(1e-4, 9e-4, 3))
        zmid = (z0 + x / 10.0 ** (3 + om[2])) * (1.0 - BETA * dt)
        mid = (0.0, 0.0, zmid)
        # the reading: mu from old alpha and old Omega ...
        mu_new = tuple((mu[i] + rb(alpha[i], om[i])) % 3 for i in range(3))
        # ... alpha from r with the new mu, before r += a'
        a_new = tuple(mid[mu_new[i]] for i in range(3))
        if len(set(mu_new)) < 2 or 2 not in mu_new:
            continue  # want alpha read from z and from 0, so a' shows
        # misreadings that must predict something else: mu moved with the
        # new alpha, alpha re-read with the old mu
        mu_with_new_alpha = tuple((mu[i] + rb(mid[mu[i]], om[i])) % 3 for i in range(3))
        if mu_with_new_alpha == mu_new or tuple(mid[m] for m in mu) == a_new:
            continue
        out.append(dict(alpha=alpha, mu=mu, om=om, x=x, z0=z0, ap=ap, zmid=zmid,
                        mu_new=mu_new, a_new_closed=a_new))
    return out


def test_step3_order_against_closed_form(prm):
    for c in _step3_cases(prm, 40):
        k = key(aprime=c["ap"])
        st = state((0.0, 0.0, c["z0"]), c["alpha"], c["mu"], c["om"])
        y = O.step_byte(k, st, c["x"], O.ENCRYPT, prm)
        alpha, mu, om, ap = c["alpha"], c["mu"], c["om"], c["ap"]
        # Step 1 with the old alpha_1, alpha_2 at the old Omega_1, Omega_2
        assert y == (c["x"] + rb(alpha[0], om[0]) + rb(alpha[1], om[1])) % 256
        # mu moved with the old alpha and the old Omega
        assert tuple(st.mu) == c["mu_new"], c
        # alpha re-read with the new mu from the state after F and before
        # r += a': 0 exactly on x and y, the decayed z otherwise
        for i in range(3):
            if c["mu_new"][i] == 2:
                assert close(st.alpha[i], c["zmid"]), (i, st.alpha[i], c["zmid"])
                assert not close(st.alpha[i], c["zmid"] + ap[2], 1e-9)
            else:
                assert st.alpha[i] == 0.0, (i, st.alpha[i])
        # Omega moved with the new alpha (the value now in the state) and the
        # old Omega; the old alpha would give another value in these cases
        want_om = tuple((om[i] + rb(st.alpha[i], om[i])) % 4 for i in range(3))
        assert tuple(st.omega) == want_om, c
        # r += a' came last: x and y are exactly a'_1 and a'_2
        assert st.r[0] == ap[0] and st.r[1] == ap[1]
        assert close(st.r[2], c["zmid"] + ap[2])


def test_step3_omega_uses_new_alpha_not_old(prm):
    # A case where the new and old alpha give different Omega updates: the
    # oracle must follow the new one.
    found = 0
    for c in _step3_cases(prm, 200):
        k = key(aprime=c["ap"])
        st = state((0.0, 0.0, c["z0"]), c["alpha"], c["mu"], c["om"])
        O.step_byte(k, st, c["x"], O.ENCRYPT, prm)
        om = c["om"]
        new = tuple((om[i] + rb(st.alpha[i], om[i])) % 4 for i in range(3))
        old = tuple((om[i] + rb(c["alpha"][i], om[i])) % 4 for i in range(3))
        if new != old:
            found += 1
            assert tuple(st.omega) == new
    assert found >= 100


def test_decrypt_kicks_with_the_recovered_plaintext(prm):
    # Reading R16: decryption recovers P in Step 1 and Step 2 kicks with P,
    # so the trajectory is the encryption's.  Encrypt x, decrypt the result
    # from the same state: the same byte and the same new state.
    rng = np.random.default_rng(5)
    for _ in range(200):
        alpha = tuple(float(v) for v in rng.uniform(-40, 40, 3))
        mu = tuple(int(v) for v in rng.integers(0, 3, 3))
        om = tuple(int(v) for v in rng.integers(0, 4, 3))
        r0 = tuple(float(v) for v in rng.uniform(-20, 20, 3))
        k = key(aprime=tuple(float(v) for v in rng.uniform(0, 1e-3, 3)))
        x = int(rng.integers(0, 256))
        se = state(r0, alpha, mu, om)
        sd = state(r0, alpha, mu, om)
        c = O.step_byte(k, se, x, O.ENCRYPT, prm)
        p = O.step_byte(k, sd, c, O.DECRYPT, prm)
        assert p == x
        assert list(se.r) == list(sd.r) and list(se.mu) == list(sd.mu)
        assert list(se.omega) == list(sd.omega) and list(se.alpha) == list(sd.alpha)


# --------------------------------------------------------------------------
# Trajectory start (Eq. 5, Sec. 5 offset) and the warm-up (n_it)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n_warm", [0, 1, 2, 17, 3000])
def test_warm_up_length_on_z_axis(n_warm):
    # r_0 = (a' + lambda) + b eta; with a' = 0, lambda = (0, 0, z0), b = 0
    # the start is on the z-axis and n_warm Euler steps give
    # z0 (1 - beta dt)^n_warm (relative rounding <= 4 n 2^-53).  alpha is
    # read after the warm-up (reading R17): alpha = r[mu].
    z0 = 25.0
    p = O.params(lam=(0.0, 0.0, z0), n_warm=n_warm)
    st = O.block_begin(key(mu=(2, 0, 1), omega=(3, 1, 2)), 0, p)
    want = z0 * (1.0 - BETA * p.dt) ** n_warm
    assert st.r[0] == 0.0 and st.r[1] == 0.0
    assert close(st.r[2], want, 1e-11), (n_warm, st.r[2], want)
    if n_warm:
        # one step more or fewer is off by a factor (1 - beta dt)
        assert not close(st.r[2], want / (1.0 - BETA * p.dt), 1e-6)
        assert not close(st.r[2], want * (1.0 - BETA * p.dt), 1e-6)
    assert list(st.mu) == [2, 0, 1] and list(st.omega) == [3, 1, 2]
    assert st.alpha[0] == st.r[2] and st.alpha[1] == 0.0 and st.alpha[2] == 0.0


def test_warm_up_is_the_v1_n_it():
    # The v1 constants: n_it = 3000 steps before the first byte.
    p = O.params()
    assert p.n_warm == 3000
    p0 = O.params(lam=(0.0, 0.0, 10.0))
    st = O.block_begin(key(), 0, p0)
    assert close(st.r[2], 10.0 * (1.0 - BETA * 0.01) ** 3000, 1e-11)


def test_trajectory_start_point():
    # Eq. 5 and the per-part offset of Sec. 5 (reading R18), before any
    # Euler step: r_j = (a'_j + lambda_j) + b eta, each sum rounded once.
    p = O.params(n_warm=0, lam=(1.0, -2.0, 20.0))
    ap = (1.2849e-4, 1.3363e-4, 1.3877e-4)
    for b in (0, 1, 5, 1 << 20):
        st = O.block_begin(key(aprime=ap), b, p)
        for j in range(3):
            assert st.r[j] == (ap[j] + p.lam[j]) + b * 2.0 ** -24, (b, j)


# --------------------------------------------------------------------------
# Fig. 1 (Sec. 3.1): digit statistics of the trajectory coordinates
# --------------------------------------------------------------------------

def _decimal_counts(vals):
    """Expected Fig. 1 counts of coordinate values from their exact decimal
    expansion: trunc(v) + 64 (clamped), floor(|v| 10^(2j+2)) mod 100 for the
    digit pairs 1-2, 3-4, 5-6; |v| >= 2^31 or NaN out of range.  Returns the
    counts and whether a value's scaled magnitude lies within one rounding
    error (|t| 2^-52) below an integer, where the binary64 product may reach it."""
    from decimal import Decimal, ROUND_DOWN, ROUND_FLOOR
    ip = np.zeros((3, 128), np.uint64)
    dg = np.zeros((3, 3, 100), np.uint64)
    oor = np.zeros(3, np.uint64)
    near = False
    for c, v in vals:
        if not (abs(v) < 2.0 ** 31):
            oor[c] += 1
            continue
        d = Decimal(v)  # exact binary value
        ip[c][min(127, max(0, int(d.to_integral_value(ROUND_DOWN)) + 64))] += 1
        a = abs(d)
        for j in range(3):
            t = a * (Decimal(10) ** (2 * j + 2))
            f = t.to_integral_value(ROUND_FLOOR)
            # rounding the product to nearest can only lift it to the next
            # integer when it lies just below one
            if (f + 1 - t) <= t * Decimal(2) ** -52:
                near = True
            dg[c][j][int(f) % 100] += 1
    return ip, dg, oor, near


def test_fig1_digit_counts_follow_the_decimal_expansion():
    # Frozen dynamics (F = identity) and a zero byte (no kick): the state the
    # oracle counts after the Euler step is exactly the state set by hand.
    p = O.params(sigma=0.0, rho=0.0, beta=0.0, dt=0.0)
    rng = np.random.default_rng(77)
    cases = [(-0.0, 12.3456789, 63.99), (-64.5, 127.25, -1e-7), (float("nan"), 2.0 ** 31, -2.0 ** 31),
             (0.005, 0.995, 99.999999), (-17.000001, 1e9, -3.5)]
    cases += [tuple(float(v) for v in rng.uniform(-70, 70, 3)) for _ in range(300)]
    cases += [tuple(float(v) for v in rng.standard_normal(3) * 10 ** rng.uniform(-4, 9, 3))
              for _ in range(300)]
    stats = O.Stats()
    vals, skipped = [], 0
    for r in cases:
        want = _decimal_counts([(c, r[c]) for c in range(3)])
        if want[3]:
            skipped += 1  # within one rounding of a digit boundary
            continue
        st = state(r, (0.0, 0.0, 0.0), (0, 1, 2), (0, 0, 0))
        O.step_byte(key(), st, 0, O.ENCRYPT, p, stats)
        vals += [(c, r[c]) for c in range(3)]
    assert skipped < 20 and len(vals) >= 3 * 580
    ip, dg, oor = stats.digit_arrays()
    want_ip, want_dg, want_oor, _ = _decimal_counts(vals)
    assert np.array_equal(ip, want_ip)
    assert np.array_equal(dg, want_dg)
    assert np.array_equal(oor, want_oor)
    assert int(stats.steps) == len(vals) // 3


def test_fig1_shape_on_a_v1_trajectory():
    # Fig. 1: the integer parts of the coordinates stay in a short range and
    # the digit pairs 3-4 and 5-6 are close to uniform.
    import scipy.stats as ss
    from paper_1201_3114_gb300 import synth
    prm = O.params()
    key_ = O.key_schedule("123456", prm)
    n = 1 << 19
    P = synth.uniform_bytes(3, n)
    Cb = np.zeros(O.ciphertext_len(n, prm=prm), np.uint8)
    st = O.Stats()
    O.encrypt_blocks(key_, P, n, Cb, 0, O.nblocks(n, prm=prm), prm, st)
    ip, dg, oor = st.digit_arrays()
    assert int(oor.sum()) == 0
    for c in range(3):
        used = np.flatnonzero(ip[c])
        assert used.size and used.max() - used.min() < 64, c  # |v| stays below ~50
        assert int(ip[c].sum()) == int(st.steps)
        for j in (1, 2):
            assert ss.chisquare(dg[c][j].astype(float)).pvalue > 1e-4, (c, j)


def test_step3_cyclic_alpha_index_profile(prm):
    # The other reading of Step 3's alpha index [(i+2) mod 3]+1: with 0-based
    # i (omega_alpha_shift = 1) Omega_1 moves with alpha_3, Omega_2 with
    # alpha_1 and Omega_3 with alpha_2 (the new alphas, the old Omegas).
    p = O.params(omega_alpha_shift=1)
    n_diff = 0
    for c in _step3_cases(prm, 60):
        st = state((0.0, 0.0, c["z0"]), c["alpha"], c["mu"], c["om"])
        O.step_byte(key(aprime=c["ap"]), st, c["x"], O.ENCRYPT, p)
        om = c["om"]
        a = [st.alpha[i] for i in range(3)]
        want = tuple((om[i] + rb(a[(i + 2) % 3], om[i])) % 4 for i in range(3))
        ident = tuple((om[i] + rb(a[i], om[i])) % 4 for i in range(3))
        assert tuple(st.omega) == want
        n_diff += want != ident
        assert tuple(st.mu) == c["mu_new"]  # mu and alpha as in the default reading
    assert n_diff >= 20


def test_both_alpha_index_readings_lock():
    # The cyclic reading does not avoid the (mu, Omega) lock: once all three
    # components share mu and Omega, their alphas coincide and every update
    # rule that treats the components alike keeps them equal, whatever the
    # alpha index.  Under both readings every part of a v1 run reaches that
    # triple lock within a few dozen bytes, after which C - P = 2 R is even.
    P = np.zeros(4096, np.uint8)
    for shift in (0, 1):
        prm = O.params(omega_alpha_shift=shift)
        key_ = O.key_schedule("123456", prm)
        st = O.block_begin(key_, 0, prm)
        locked_at = None
        for i in range(400):
            O.step_byte(key_, st, 0, O.ENCRYPT, prm)
            triple = len(set(st.mu)) == 1 and len(set(st.omega)) == 1
            if locked_at is None and triple:
                locked_at = i
            if locked_at is not None:
                assert triple, (shift, i)  # absorbing
        assert locked_at is not None and locked_at < 100, (shift, locked_at)
        c = O.encrypt("123456", P, O.PARALLEL, prm)[:4096].astype(int)
        assert np.all((c[128:] - P[128:].astype(int)) % 2 == 0), shift
