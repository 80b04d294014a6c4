// softfp64.cuh -- IEEE-754 binary64 round-to-nearest-even arithmetic on the
// 32-bit integer pipe.
//
// GB300 executes binary64 add/multiply at about 1/38 of its 32-bit integer
// rate.  These functions compute the correctly rounded binary64 result of
// an operation from the operands' bit patterns with integer instructions
// only, so a kernel can split its binary64 work between the two pipes.  Each
// function handles the common case (normal operands, normal result) in
// integer arithmetic and defers every other case (zeros, subnormals,
// infinities, NaNs, results near overflow or underflow) to the hardware
// instruction, so the result is bit-identical to the hardware's for every
// input.  The rounding rule is the textbook one (IEEE 754-2019 Sec. 4.3.1):
// keep the leading 53 bits, round up when the discarded part exceeds half an
// ulp, or equals half an ulp and the kept part is odd.
//
// Representation: x = (-1)^s * M * 2^(e - 1075) for a normal x, with the
// biased exponent e in [1, 2046] and the 53-bit significand M in
// [2^52, 2^53).  Results are packed as s | (E - 1) << 52 + q with q in
// [2^52, 2^53]: the hidden bit of q adds one to the exponent field, and a
// rounding carry to q = 2^53 adds one more, which is exactly the binade step.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lc {
namespace sfp {

constexpr uint64_t kSign = 0x8000000000000000ull;
constexpr uint64_t kFrac = 0x000FFFFFFFFFFFFFull;
constexpr uint64_t kHidden = 0x0010000000000000ull;

__device__ __forceinline__ uint64_t bits(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ double from_bits(uint64_t b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ uint32_t bexp(uint64_t b) { return (uint32_t)(b >> 52) & 0x7FFu; }

// Hardware fallbacks, kept out of line on purpose: a short inline branch is
// turned into predicated instructions, and a predicated-off binary64
// instruction still occupies the narrow FP64 pipe.  Behind a call it runs
// only when the rare case really happens.
static __device__ __noinline__ double hw_mul(double a, double b) { return __dmul_rn(a, b); }
static __device__ __noinline__ double hw_add(double a, double b) { return __dadd_rn(a, b); }
static __device__ __noinline__ uint32_t hw_floor13_lo32(double a) {
  return (uint32_t)(uint64_t)__double2ll_rd(__dmul_rn(a, 1e13));
}

__device__ __forceinline__ uint32_t lo32(double x) { return (uint32_t)__double2loint(x); }
__device__ __forceinline__ uint32_t hi32(double x) { return (uint32_t)__double2hiint(x); }
__device__ __forceinline__ double pack(uint32_t hi, uint32_t lo) { return __hiloint2double((int)hi, (int)lo); }

// x * (K * 2^E) for a small odd integer K (3 <= K < 256): the product M * K
// has at most 61 bits and is rounded to 53 by one shift.
template <uint32_t K, int E>
__device__ __forceinline__ double mul_small(double x) {
  static_assert(K >= 3 && K < 256 && (K & 1u), "K must be a small odd integer");
  constexpr uint32_t kb = (K < 4) ? 2 : (K < 8) ? 3 : (K < 16) ? 4 : (K < 32) ? 5 : (K < 64) ? 6 : (K < 128) ? 7 : 8;
  const uint32_t xl = lo32(x), xh = hi32(x);
  const uint32_t e = (xh >> 20) & 0x7FFu;
  // fast path: normal x and a normal result (margin for the binade step)
  if (e - 1u >= 2045u - (uint32_t)E - kb) return hw_mul(x, (double)K * (double)(1ll << E));
  const uint32_t m1 = (xh & 0xFFFFFu) | 0x100000u;
  const uint64_t plo = (uint64_t)xl * K;                 // m0 K
  const uint32_t p0 = (uint32_t)plo;
  const uint32_t p1 = m1 * K + (uint32_t)(plo >> 32);   // P = p1:p0 < 2^61
  // P has 52 + kb or 53 + kb bits; shift so that 53 remain.
  const uint32_t sh = kb - 1u + ((p1 >> (20u + kb)) & 1u);
  uint32_t q0 = __funnelshift_r(p0, p1, sh);
  uint32_t q1 = p1 >> sh;
  const uint32_t rem = p0 & ((1u << sh) - 1u);
  const uint32_t half = 1u << (sh - 1u);
  const uint32_t up = (rem > half || (rem == half && (q0 & 1u))) ? 1u : 0u;
  q0 += up;
  q1 += (q0 < up) ? 1u : 0u;
  // biased exponent of the result: e + E + sh; the hidden bit of q adds one
  const uint32_t hi = (xh & 0x80000000u) + ((e + (uint32_t)E + sh - 1u) << 20) + q1;
  return pack(hi, q0);
}

// Low 32 bits of floor(RN(a * 10^13)) as a two's complement integer, the
// value cvt.rmi.s64.f64 gives (saturating, NaN -> 0).  10^13 = 5^13 * 2^13
// and 5^13 = 1220703125 < 2^31, so M * 5^13 has 83 or 84 bits; rounding it
// to 53 bits is the binary64 product, and the floor then drops the bits
// below the binary point.
__device__ __forceinline__ uint32_t floor_scaled_lo32(double a) {
  constexpr uint32_t kFive13 = 1220703125u;
  const uint32_t xl = lo32(a), xh = hi32(a);
  const uint32_t e = (xh >> 20) & 0x7FFu;
  // 2^-43 <= |a| < 2^36; the value's own range is checked after rounding
  if (e - 980u > 78u) return hw_floor13_lo32(a);
  const uint32_t m1 = (xh & 0xFFFFFu) | 0x100000u;
  const uint64_t p0 = (uint64_t)xl * kFive13;                       // < 2^63
  const uint64_t mid = (uint64_t)m1 * kFive13 + (p0 >> 32);         // < 2^53
  // P = mid:w0 (84 bits): w1 = low(mid), w2 = high(mid)
  const uint32_t w0 = (uint32_t)p0, w1 = (uint32_t)mid, w2 = (uint32_t)(mid >> 32);
  const uint32_t top = (w2 >> 19) & 1u;  // P >= 2^83
  const uint32_t sh = 30u + top;         // q = P >> sh has 53 bits
  uint32_t q0 = __funnelshift_r(w0, w1, sh);
  uint32_t q1 = __funnelshift_r(w1, w2, sh);
  const uint32_t rem = w0 & ((1u << sh) - 1u);
  const uint32_t half = 1u << (sh - 1u);
  const uint32_t up = (rem > half || (rem == half && (q0 & 1u))) ? 1u : 0u;
  q0 += up;
  q1 += (q0 < up) ? 1u : 0u;
  // RN(a 1e13) = q 2^-d with d = 1062 - e - sh fraction bits
  const uint32_t d = 1062u - e - sh;
  if (d - 1u > 52u) return hw_floor13_lo32(a);  // d outside [1, 53]
  // integer part (low 32 bits) and whether a fraction remains
  uint32_t ip, frac;
  if (d < 32u) {
    ip = __funnelshift_r(q0, q1, d);
    frac = q0 << (32u - d);
  } else {
    ip = q1 >> (d - 32u);
    frac = q0 | (d > 32u ? (q1 << (64u - d)) : 0u);
  }
  if (xh & 0x80000000u) return 0u - ip - (frac != 0u ? 1u : 0u);
  return ip;
}

// The integer path of RN(a * b), from the operands' fields: a's low and high
// words, b's low word, b's significand above bit 32 with its hidden bit, the
// product's biased exponent if it stays in [1, 2), and the product's sign
// bit.  The caller has checked that a, b and the result are normal.
__device__ __forceinline__ double dmul_fields(uint32_t xl, uint32_t xh, uint32_t yl, uint32_t b1, uint32_t er,
                                              uint32_t sign) {
  const uint32_t a1 = (xh & 0xFFFFFu) | 0x100000u;
  const uint64_t p00 = (uint64_t)xl * yl;
  const uint64_t mid = (uint64_t)xl * b1 + (uint64_t)a1 * yl;  // < 2^54
  const uint64_t p11 = (uint64_t)a1 * b1;                      // < 2^42
  // P = p00 + mid 2^32 + p11 2^64 = w3:w2:w1:w0, in [2^104, 2^106)
  const uint64_t s1 = (p00 >> 32) + (uint32_t)mid;
  const uint64_t s2 = (s1 >> 32) + (mid >> 32) + p11;
  const uint32_t w0 = (uint32_t)p00, w1 = (uint32_t)s1;
  const uint32_t w2 = (uint32_t)s2, w3 = (uint32_t)(s2 >> 32);
  const uint32_t top = (w3 >> 9) & 1u;  // P >= 2^105
  const uint32_t s = 20u + top;         // drop 52 + top bits: w0 and s bits of w1
  uint32_t q0 = __funnelshift_r(w1, w2, s);
  uint32_t q1 = __funnelshift_r(w2, w3, s);
  const uint32_t guard = (w1 >> (s - 1u)) & 1u;
  const uint32_t sticky = w0 | (w1 << (33u - s));
  const uint32_t up = guard & ((sticky != 0u) | (q0 & 1u));
  q0 += up;
  q1 += (q0 < up) ? 1u : 0u;
  const uint32_t hi = sign + ((er + top - 1u) << 20) + q1;
  return pack(hi, q0);
}

// RN(a * b) for two normal operands with a normal result.
__device__ __forceinline__ double dmul(double a, double b) {
  const uint32_t xl = lo32(a), xh = hi32(a), yl = lo32(b), yh = hi32(b);
  const uint32_t ea = (xh >> 20) & 0x7FFu, eb = (yh >> 20) & 0x7FFu;
  const uint32_t er = ea + eb - 1023u;  // biased exponent if the product stays in [1, 2)
  if (ea - 1u >= 2046u || eb - 1u >= 2046u || er - 1u >= 2044u) return hw_mul(a, b);
  return dmul_fields(xl, xh, yl, (yh & 0xFFFFFu) | 0x100000u, er, (xh ^ yh) & 0x80000000u);
}

// RN(a * C) for a compile-time constant C given by its bit pattern CB (a
// positive normal number): dmul with the constant's fields folded in.
template <uint64_t CB>
__device__ __forceinline__ double dmul_const(double a) {
  constexpr uint32_t yl = (uint32_t)CB;
  constexpr uint32_t b1 = (uint32_t)((CB >> 32) & 0xFFFFFull) | 0x100000u;
  constexpr uint32_t eb = (uint32_t)(CB >> 52) & 0x7FFu;
  static_assert(eb >= 1u && eb <= 2046u && (CB >> 63) == 0, "a positive normal constant");
  const uint32_t xl = lo32(a), xh = hi32(a);
  const uint32_t ea = (xh >> 20) & 0x7FFu;
  const uint32_t er = ea + eb - 1023u;
  if (ea - 1u >= 2046u || er - 1u >= 2044u) return hw_mul(a, from_bits(CB));
  return dmul_fields(xl, xh, yl, b1, er, xh & 0x80000000u);
}

// The adders' shared core.  add_aligned: X1:X0 + Y or X1:X0 - Y (sub = 1),
// where Y is Y1:Y0 shifted right by the gap d < 32 with every bit shifted
// out folded into its bit 0 (sticky).  add_round_pack: R is that sum, its
// leading bit at 63 - lz (lz <= 2); keep the 53 bits from the leading one,
// round half to even, and pack with the sign bit and the biased exponent ex
// of the larger operand.
__device__ __forceinline__ uint64_t add_aligned(uint32_t X1, uint32_t X0, uint32_t Y1, uint32_t Y0, uint32_t d,
                                                uint32_t sub) {
  const uint32_t s0 = __funnelshift_r(Y0, Y1, d), s1 = Y1 >> d;
  const uint32_t lost = Y0 & ((1u << d) - 1u);
  // X + Y, or X - Y as X + ~Y + 1
  const uint32_t m = 0u - sub;
  const uint32_t t0 = (s0 | (lost != 0u ? 1u : 0u)) ^ m, t1 = s1 ^ m;
  return ((((uint64_t)X1 << 32) | X0) + (((uint64_t)t1 << 32) | t0)) + sub;
}
__device__ __forceinline__ double add_round_pack(uint64_t R, uint32_t ex, uint32_t sign) {
  // leading bit at 63 - lz; the result's biased exponent is ex + 1 - lz
  const uint32_t lz = __clz((uint32_t)(R >> 32));
  const uint32_t rp = 11u - lz;  // bits below the last kept place
  const uint32_t last = ((uint32_t)R >> rp) & 1u;
  const uint64_t T = R + ((1u << (rp - 1u)) - 1u + last);
  const uint32_t T1 = (uint32_t)(T >> 32), T0 = (uint32_t)T;
  const uint32_t q0 = __funnelshift_r(T0, T1, rp), q1 = T1 >> rp;
  // q has its hidden bit at 2^52 (2^53 after a rounding carry), which
  // supplies the last 1 of the exponent field (or steps to the next binade)
  return pack(sign + ((ex - lz) << 20) + q1, q0);
}

// RN(a + b) for two normal operands (either sign) with a normal result.
// Subtraction of operands whose exponents differ by at most one can cancel
// many leading bits; that case, and exponent gaps of 32 or more (where b
// only affects the rounding), are rare in the cipher and go to the hardware.
//
// The significands are placed at bits 62..10 of 64-bit words, leaving ten
// bits below the last place.  The smaller operand is shifted right by the
// gap d < 32 and any bits shifted out are folded into its bit 0 (sticky):
// with ten spare bits the folded value and the exact one round the same
// way.  The sum then has its leading bit at 63, 62 or 61, so rounding keeps
// the 53 bits from the leading one: round-half-even by adding half an ulp
// minus one plus the last kept bit, then truncating.
__device__ __forceinline__ double dadd(double a, double b) {
  const uint32_t ah = hi32(a), al = lo32(a), bh = hi32(b), bl = lo32(b);
  // order by magnitude (high words suffice: equal high words mean equal
  // exponents, where the order does not matter or the hardware is used)
  const uint32_t mah = ah & 0x7FFFFFFFu, mbh = bh & 0x7FFFFFFFu;
  const bool sw = mah < mbh;
  const uint32_t xh = sw ? bh : ah, xl = sw ? bl : al;
  const uint32_t yh = sw ? ah : bh, yl = sw ? al : bl;
  const uint32_t ex = max(mah, mbh) >> 20, ey = min(mah, mbh) >> 20;
  const uint32_t d = ex - ey;
  const uint32_t sub = (ah ^ bh) >> 31;
  // fast path: y normal, no overflow past the top binade, gap < 32, and a
  // subtraction only with gap >= 2 (at most one leading bit cancels)
  if (ey == 0u || ex > 2045u || d > 31u || (sub != 0u && d < 2u)) return hw_add(a, b);
  const uint32_t xm = (xh & 0xFFFFFu) | 0x100000u, ym = (yh & 0xFFFFFu) | 0x100000u;
  const uint32_t X1 = __funnelshift_l(xl, xm, 10), X0 = xl << 10;
  const uint32_t Y1 = __funnelshift_l(yl, ym, 10), Y0 = yl << 10;
  return add_round_pack(add_aligned(X1, X0, Y1, Y0, d, sub), ex, xh & 0x80000000u);
}

__device__ __forceinline__ double dsub(double a, double b) { return dadd(a, -b); }

// RN(x + a) where x is the larger operand in magnitude, by an exponent gap
// d of 1..31 (2..31 when the signs differ, so at most one leading bit
// cancels): dadd with the operand order known, so no comparison or swap.
// kXPos / kAPos: the caller expects x / a to be positive; the fast path then
// checks that sign and leaves it out of the sign logic.  Every other case
// (an operand zero, subnormal or not finite, x in the top binade, a gap
// outside the range, an operand of the other sign) goes to the hardware,
// except x + 0 = x for a normal x.
template <bool kXPos, bool kAPos>
__device__ __forceinline__ double dadd_small(double x, double a) {
  const uint32_t xh = hi32(x), xl = lo32(x), ah = hi32(a), al = lo32(a);
  // with the sign bit kept, a negative operand gives an exponent >= 2048,
  // which fails the range checks below
  const uint32_t ex = kXPos ? xh >> 20 : (xh >> 20) & 0x7FFu;
  const uint32_t ea = kAPos ? ah >> 20 : (ah >> 20) & 0x7FFu;
  const uint32_t sub = (kXPos ? 0u : xh >> 31) ^ (kAPos ? 0u : ah >> 31);
  const uint32_t d = ex - ea;
  // d in [1 + sub, 31]; unsigned wrap-around sends d <= sub to the hardware
  const bool fast = ea != 0u && ex <= 2045u && d - 1u - sub <= 30u - sub;
  if (!fast) {
    // x + 0 = x for a normal x (the cipher's kick adds +0 for a zero byte)
    if (((ah & 0x7FFFFFFFu) | al) == 0u && ((xh >> 20) & 0x7FFu) - 1u <= 2045u) return x;
    return hw_add(x, a);
  }
  const uint32_t xm = (xh & 0xFFFFFu) | 0x100000u, am = (ah & 0xFFFFFu) | 0x100000u;
  const uint32_t X1 = __funnelshift_l(xl, xm, 10), X0 = xl << 10;
  const uint32_t Y1 = __funnelshift_l(al, am, 10), Y0 = al << 10;
  return add_round_pack(add_aligned(X1, X0, Y1, Y0, d, sub), ex, xh & 0x80000000u);
}

}  // namespace sfp
}  // namespace lc
