"""The integer-pipe binary64 routines against the hardware instructions.

Each routine must return exactly the bits of the hardware's
round-to-nearest-even result (or cvt.rmi.s64.f64's low word) for every
input: normal operands in the cipher's range, every exponent gap for the
adder, exact cancellation, operands whose results are exact ties, zeros,
subnormals, infinities, NaNs and values near overflow and underflow (the
latter cases must take the hardware fallback)."""
import numpy as np
import pytest

from paper_1201_3114_gb300 import lc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
N = 1 << 21


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def _specials():
    vals = [0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, -2.2250738585072014e-308,
            2.225073858507201e-308, 1.7976931348623157e308, -1.7976931348623157e308,
            float("inf"), float("-inf"), float("nan"), 1.0, -1.0, 0.5, 2.0 ** -1022, 2.0 ** 1023,
            2.0 ** -1074 * 3, 1e-300, 1e300, 4.9e-309]
    return np.array(vals, dtype=np.float64)


def _operands(rng, n):
    """Mixture: raw bit patterns, cipher-range values, wide exponents,
    small-significand values (ties), dyadic integers."""
    k = n // 6
    raw = rng.integers(0, 2 ** 63, k, dtype=np.uint64) | (rng.integers(0, 2, k, dtype=np.uint64) << np.uint64(63))
    lorenz = rng.uniform(-80, 80, k) * rng.choice([1.0, 1e-2, 1e-4, 1e3], k)
    wide = np.ldexp(rng.uniform(1, 2, k), rng.integers(-1080, 1080, k)) * rng.choice([-1.0, 1.0], k)
    small_sig = rng.integers(1, 256, k).astype(np.float64) * np.ldexp(1.0, rng.integers(-40, 40, k))
    small_sig *= rng.choice([-1.0, 1.0], k)
    dyadic = rng.integers(-2 ** 40, 2 ** 40, k).astype(np.float64) * np.ldexp(1.0, -rng.integers(0, 60, k))
    rest = n - 5 * k
    near = rng.uniform(-1, 1, rest) * np.ldexp(1.0, rng.integers(-20, 8, rest))
    parts = [raw, _f64(lorenz), _f64(wide), _f64(small_sig), _f64(dyadic), _f64(near)]
    out = np.concatenate(parts)
    rng.shuffle(out)
    return out


def _eval(op, a, b=None):
    A = torch.from_numpy(a.view(np.int64)).cuda()
    Bt = torch.from_numpy(b.view(np.int64)).cuda() if b is not None else None
    sw = torch.empty_like(A)
    hw = torch.empty_like(A)
    lc.check(lc.lc_softfp_eval(op, A, Bt, sw, hw, a.size))
    torch.cuda.synchronize()
    return sw.cpu().numpy().view(np.uint64), hw.cpu().numpy().view(np.uint64)


def _check(op, a, b=None):
    sw, hw = _eval(op, a, b)
    bad = np.flatnonzero(sw != hw)
    if bad.size:
        i = bad[0]
        av = a[i:i + 1].view(np.float64)[0]
        bv = b[i:i + 1].view(np.float64)[0] if b is not None else None
        raise AssertionError("op %d: %d mismatches, first a=%r (%#x) b=%r sw=%#x hw=%#x"
                             % (op, bad.size, av, int(a[i]), bv, int(sw[i]), int(hw[i])))


@pytest.fixture(scope="module")
def rng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return np.random.default_rng(1234)


@pytest.mark.parametrize("op", [lc.LC_SFP_ADD, lc.LC_SFP_SUB, lc.LC_SFP_MUL, lc.LC_SFP_ADD_KICK, lc.LC_SFP_ADD_Z])
def test_two_operand_routines_random(rng, op):
    a = _operands(rng, N)
    b = _operands(rng, N)
    _check(op, a, b)
    # operands against every special value
    s = _f64(_specials())
    aa = np.repeat(s, s.size)
    bb = np.tile(s, s.size)
    _check(op, aa, bb)
    x = _operands(rng, 4096)
    _check(op, np.repeat(s, x.size), np.tile(x, s.size))
    _check(op, np.tile(x, s.size), np.repeat(s, x.size))


def test_adder_every_exponent_gap_and_cancellation(rng):
    n = 1 << 20
    a = np.ldexp(rng.uniform(1, 2, n), rng.integers(-30, 30, n)) * rng.choice([-1.0, 1.0], n)
    gap = rng.integers(0, 70, n)
    b = np.ldexp(rng.uniform(1, 2, n), np.frexp(a)[1] - 1 - gap) * rng.choice([-1.0, 1.0], n)
    _check(lc.LC_SFP_ADD, _f64(a), _f64(b))
    _check(lc.LC_SFP_SUB, _f64(a), _f64(b))
    # near-cancellation: b = -a perturbed in its last bits
    ai = _f64(a)
    pert = ai ^ rng.integers(0, 1 << 12, n, dtype=np.uint64)
    _check(lc.LC_SFP_ADD, ai, pert ^ np.uint64(1 << 63))
    _check(lc.LC_SFP_SUB, ai, pert)
    # exact halfway sums: 1 + 2^-53 style ties at many scales
    k = rng.integers(-40, 40, n)
    t = np.ldexp(rng.integers(2 ** 52, 2 ** 53, n).astype(np.float64), k - 52)
    h = np.ldexp(1.0, k - 53) * rng.choice([1.0, 3.0, -1.0, -3.0], n)
    _check(lc.LC_SFP_ADD, _f64(t), _f64(h))


def test_known_order_adders(rng):
    """The kick's adder (a larger than b >= 0) and the z update's (a > 0
    larger than b): the cipher's own operands, every gap with both signs,
    near-cancellation, exact ties, and operands in the wrong order or with
    the wrong sign (which must take the hardware path)."""
    n = 1 << 20
    # the kick: a coordinate and Theta = P / 10^(3 + Omega)
    x = rng.uniform(-60, 60, n)
    P = rng.integers(0, 256, n).astype(np.float64)
    theta = P / np.array([1e3, 1e4, 1e5, 1e6])[rng.integers(0, 4, n)]
    _check(lc.LC_SFP_ADD_KICK, _f64(x), _f64(theta))
    # the z update: z and dt dz of either sign
    z = rng.uniform(0.5, 50, n)
    dz = rng.uniform(-6, 6, n)
    _check(lc.LC_SFP_ADD_Z, _f64(z), _f64(dz))
    a = np.ldexp(rng.uniform(1, 2, n), rng.integers(-30, 30, n))
    gap = rng.integers(-3, 40, n)
    b = np.ldexp(rng.uniform(1, 2, n), np.frexp(a)[1] - 1 - gap)
    sa, sb = rng.choice([-1.0, 1.0], n), rng.choice([-1.0, 1.0], n)
    for op in (lc.LC_SFP_ADD_KICK, lc.LC_SFP_ADD_Z):
        _check(op, _f64(a), _f64(b))
        _check(op, _f64(a * sa), _f64(b))
        _check(op, _f64(a), _f64(b * sb))
        _check(op, _f64(a * sa), _f64(b * sb))
        # near-cancellation and exact halfway sums
        ai = _f64(a)
        pert = ai ^ rng.integers(0, 1 << 12, n, dtype=np.uint64)
        _check(op, ai, pert ^ np.uint64(1 << 63))
        k = rng.integers(-40, 40, n)
        t = np.ldexp(rng.integers(2 ** 52, 2 ** 53, n).astype(np.float64), k - 52)
        h = np.ldexp(1.0, k - 53) * rng.choice([1.0, 3.0, -1.0, -3.0], n)
        _check(op, _f64(t), _f64(h))
        _check(op, _f64(t), _f64(np.abs(h)))
        # zero addends: x + 0 = x, and -0 + 0 = +0
        _check(op, _f64(np.r_[x, -0.0, 0.0, 5e-324]), _f64(np.zeros(n + 3)))
        _check(op, _f64(np.r_[x, -0.0, 0.0, 5e-324]), _f64(np.full(n + 3, -0.0)))


def _const_ties(rng, n, c):
    """a whose product with the constant c lies exactly halfway between two
    binary64 values: with c's significand C odd, M = 2^52 + (2^51 C^-1 mod
    2^52) gives a 105-bit M C whose low 52 bits are 2^51."""
    C = (int(np.float64(c).view(np.uint64)) & ((1 << 52) - 1)) | 1 << 52
    M = (1 << 52) | ((pow(C, -1, 1 << 52) << 51) % (1 << 52))
    assert (M * C).bit_length() == 105 and (M * C) % (1 << 52) == 1 << 51
    e = rng.integers(-1000, 1000, n)
    return np.ldexp(float(M), e - 52) * rng.choice([-1.0, 1.0], n)


def test_small_constant_multiples(rng):
    a = _operands(rng, N)
    s = _f64(_specials())
    for op in (lc.LC_SFP_MUL10, lc.LC_SFP_MUL28, lc.LC_SFP_MULDT, lc.LC_SFP_MULBETA):
        _check(op, a)
        _check(op, s)
    # halfway products and results next to the normal range's ends
    _check(lc.LC_SFP_MULDT, _f64(_const_ties(rng, 1 << 16, 0.01)))
    _check(lc.LC_SFP_MULBETA, _f64(_const_ties(rng, 1 << 16, 8.0 / 3.0)))
    edge = np.ldexp(rng.uniform(1, 2, 1 << 18), rng.choice(np.r_[-1030:-1010, 1015:1031], 1 << 18))
    _check(lc.LC_SFP_MULDT, _f64(edge))
    _check(lc.LC_SFP_MULBETA, _f64(edge))


def test_general_multiply_ties(rng):
    # b with a few significant bits makes a*b land on exact halfway points often
    n = 1 << 20
    a = np.ldexp(rng.uniform(1, 2, n), rng.integers(-60, 60, n)) * rng.choice([-1.0, 1.0], n)
    b = rng.integers(1, 4096, n).astype(np.float64) * np.ldexp(1.0, rng.integers(-20, 20, n))
    _check(lc.LC_SFP_MUL, _f64(a), _f64(b))
    # the cipher's own constants
    for c in (0.01, 8.0 / 3.0, 10.0, 28.0, 1e13):
        _check(lc.LC_SFP_MUL, _f64(a), _f64(np.full(n, c)))


def _floor_ties(rng, n):
    """alpha whose product with 10^13 lies exactly halfway between two
    binary64 values: M * 5^13 = q 2^s + 2^(s-1) with s = 30 or 31."""
    five13 = 5 ** 13
    out = []
    while len(out) < n:
        s = int(rng.integers(30, 32))
        inv = pow(five13, -1, 1 << s)
        low = (inv << (s - 1)) % (1 << s)
        M = (int(rng.integers(2 ** 21, 2 ** 22)) << 31 | low) & ((1 << 53) - 1)
        if M < 2 ** 52 or (M * five13).bit_length() != 53 + s:
            continue
        e = int(rng.integers(-20, 7))
        v = float(M) * 2.0 ** (e - 52)
        out.append(v if rng.integers(0, 2) else -v)
    return np.array(out, dtype=np.float64)


def test_floor_scaled(rng):
    a = _operands(rng, N)
    _check(lc.LC_SFP_FLOOR13, a)
    _check(lc.LC_SFP_FLOOR13, _f64(_specials()))
    _check(lc.LC_SFP_FLOOR13, _f64(_floor_ties(rng, 20000)))
    # exact integers after scaling, positive and negative, and tiny values
    k = rng.integers(-2 ** 45, 2 ** 45, 1 << 18).astype(np.float64)
    _check(lc.LC_SFP_FLOOR13, _f64(k / 1e13))
    _check(lc.LC_SFP_FLOOR13, _f64(np.ldexp(rng.uniform(-1, 1, 1 << 18), rng.integers(-60, 40, 1 << 18))))
