// keysched.cpp -- host-side key schedule of the Lorenz cipher: the password
// is packed into three integers (Sec. 3.1, Eqs. 2-4), scaled into [0, 1)
// (g(x)), reduced mod 3 for mu and hashed for Omega (Eq. 7).
//
// Runs once per password; the result is cached by the context.
#include "keysched.h"

#include <math.h>
#include <string.h>

namespace lc {

namespace {

// ---------------------------------------------------------------------------
// SHA-256 (FIPS 180-4).  The round constants are the first 32 fractional
// bits of the cube roots of the first 64 primes and the initial hash the
// first 32 fractional bits of the square roots of the first 8 primes; they
// are derived here with exact integer roots instead of being typed in.
// ---------------------------------------------------------------------------

struct ShaConstants {
  uint32_t k[64];
  uint32_t h0[8];
  ShaConstants() {
    int found = 0;
    for (uint32_t c = 2; found < 64; c++) {
      bool prime = true;
      for (uint32_t d = 2; d * d <= c; d++)
        if (c % d == 0) { prime = false; break; }
      if (!prime) continue;
      // floor(cbrt(c) * 2^32) = floor(cbrt(c * 2^96))
      u128 target = (u128)c << 96;
      uint64_t lo = 0, hi = (uint64_t)1 << 40;
      while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        u128 m = mid;
        if (m * m * m <= target) lo = mid; else hi = mid;
      }
      k[found] = (uint32_t)lo;
      if (found < 8) {
        // floor(sqrt(c) * 2^32) = floor(sqrt(c * 2^64))
        u128 t2 = (u128)c << 64;
        uint64_t a = 0, b = (uint64_t)1 << 40;
        while (b - a > 1) {
          uint64_t mid = a + (b - a) / 2;
          u128 m = mid;
          if (m * m <= t2) a = mid; else b = mid;
        }
        h0[found] = (uint32_t)a;
      }
      found++;
    }
  }
};

const ShaConstants& sha_constants() {
  static const ShaConstants c;
  return c;
}

inline uint32_t ror(uint32_t v, unsigned s) { return (v >> s) | (v << (32u - s)); }

void sha_compress(uint32_t st[8], const uint8_t* p, const uint32_t* K) {
  uint32_t w[16];
  for (int i = 0; i < 16; i++)
    w[i] = (uint32_t)p[4 * i] << 24 | (uint32_t)p[4 * i + 1] << 16 |
           (uint32_t)p[4 * i + 2] << 8 | (uint32_t)p[4 * i + 3];
  uint32_t v[8];
  memcpy(v, st, sizeof v);
  for (int t = 0; t < 64; t++) {
    uint32_t wt;
    if (t < 16) {
      wt = w[t];
    } else {
      // rolling 16-word schedule
      uint32_t x15 = w[(t + 1) & 15], x2 = w[(t + 14) & 15];
      uint32_t g0 = ror(x15, 7) ^ ror(x15, 18) ^ (x15 >> 3);
      uint32_t g1 = ror(x2, 17) ^ ror(x2, 19) ^ (x2 >> 10);
      wt = w[t & 15] = w[t & 15] + g0 + w[(t + 9) & 15] + g1;
    }
    uint32_t e = v[4], a = v[0];
    uint32_t ch = (e & v[5]) ^ (~e & v[6]);
    uint32_t maj = (a & v[1]) ^ (a & v[2]) ^ (v[1] & v[2]);
    uint32_t T1 = v[7] + (ror(e, 6) ^ ror(e, 11) ^ ror(e, 25)) + ch + K[t] + wt;
    uint32_t T2 = (ror(a, 2) ^ ror(a, 13) ^ ror(a, 22)) + maj;
    memmove(v + 1, v, 7 * sizeof(uint32_t));
    v[4] += T1;
    v[0] = T1 + T2;
  }
  for (int i = 0; i < 8; i++) st[i] += v[i];
}

}  // namespace

void sha256(const uint8_t* msg, size_t len, uint8_t out[32]) {
  const ShaConstants& C = sha_constants();
  uint32_t st[8];
  memcpy(st, C.h0, sizeof st);
  size_t full = len / 64;
  for (size_t i = 0; i < full; i++) sha_compress(st, msg + 64 * i, C.k);
  uint8_t tail[128];
  memset(tail, 0, sizeof tail);
  size_t r = len - 64 * full;
  memcpy(tail, msg + 64 * full, r);
  tail[r] = 0x80;
  size_t tl = (r + 1 + 8 <= 64) ? 64 : 128;
  uint64_t bits = (uint64_t)len << 3;
  for (int i = 0; i < 8; i++) tail[tl - 1 - i] = (uint8_t)(bits >> (8 * i));
  for (size_t off = 0; off < tl; off += 64) sha_compress(st, tail + off, C.k);
  for (int i = 0; i < 32; i++) out[i] = (uint8_t)(st[i / 4] >> (24 - 8 * (i % 4)));
}

double u128_to_double(u128 v) {
  if (v == 0) return 0.0;
  int nbits = 0;
  for (u128 t = v; t; t >>= 1) nbits++;
  if (nbits <= 53) return (double)(uint64_t)v;  // exact
  int drop = nbits - 53;
  uint64_t keep = (uint64_t)(v >> drop);  // 53 significant bits
  u128 rest = v - ((u128)keep << drop);
  u128 half = (u128)1 << (drop - 1);
  if (rest > half || (rest == half && (keep & 1u))) {
    keep += 1;
    if (keep == ((uint64_t)1 << 53)) {  // carried into a new bit
      keep >>= 1;
      drop += 1;
    }
  }
  return ldexp((double)keep, drop);  // exact scaling by a power of two
}

double pow10_rn(int e) {
  u128 v = 1;
  for (int i = 0; i < e; i++) v *= 10u;
  return u128_to_double(v);
}

bool params_valid(const lc_params& p) {
  if (!(p.dt == p.dt) || !(p.sigma == p.sigma) || !(p.rho == p.rho) || !(p.beta == p.beta))
    return false;
  if (p.steps_per_byte < 1 || p.steps_per_byte > 4096) return false;
  for (int i = 0; i < 3; i++)
    if (p.k[i] < 1 || p.k[i] > 8) return false;
  if (p.block_len < 16 || p.block_len > (1u << 24) || (p.block_len % 16) != 0) return false;
  if (p.tag_len < 1 || p.tag_len > 8) return false;
  if (p.omega_alpha_shift > 1 || p.reserved != 0) return false;
  return true;
}

lc_status key_schedule(const lc_params& p, const uint8_t* pw, size_t n, HostKey* out) {
  if (pw == nullptr || n < 1 || n > 32) return LC_ERR_PASSWORD;
  const size_t L = n / 3, rem = n % 3;

  // Placement of each password byte (Eqs. 2-4): component and byte position.
  // a_1 takes the first L bytes, shifted up one byte when a leftover
  // character (the (3L+1)-th) occupies its lowest byte; a_2 likewise with
  // the (3L+2)-th character when two are left over; a_3 the third L bytes.
  u128 a[3] = {0, 0, 0};
  auto put = [&](int comp, size_t pos, uint8_t byte) { a[comp] |= (u128)byte << (8 * pos); };
  for (size_t j = 0; j < L; j++) {
    put(0, j + (rem != 0 ? 1 : 0), pw[j]);
    put(1, j + (rem == 2 ? 1 : 0), pw[L + j]);
    put(2, j, pw[2 * L + j]);
  }
  if (rem >= 1) put(0, 0, pw[3 * L]);
  if (rem == 2) put(1, 0, pw[3 * L + 1]);

  // g(x) = x / 10^D, D = ceil(log10 2^(8(L+1))): the least D with
  // 10^D >= 2^(8(L+1)).
  const unsigned bits = 8u * (unsigned)(L + 1);
  uint32_t D = 0;
  {
    u128 pw10 = 1;
    const u128 lim = (u128)1 << bits;
    while (pw10 < lim) { pw10 *= 10u; D++; }
  }
  const double tenD = pow10_rn((int)D);

  // a mod 3 from the byte sum (256 = 1 mod 3).
  uint32_t m3[3];
  for (int c = 0; c < 3; c++) {
    uint32_t s = 0;
    for (int byte = 0; byte < 16; byte++) s += (uint32_t)(uint8_t)(a[c] >> (8 * byte));
    m3[c] = s % 3u;
  }

  HostKey K;
  for (int c = 0; c < 3; c++) {
    K.a[c] = a[c];
    K.aprime[c] = u128_to_double(a[c]) / tenD;
  }
  K.L = (uint32_t)L;
  K.D = D;
  K.mu[0] = (m3[0] + m3[1] + m3[2]) % 3u;
  K.mu[1] = (m3[0] * m3[1] + m3[2]) % 3u;
  K.mu[2] = (m3[0] + m3[1] * m3[2]) % 3u;

  // Eq. 7: Omega_i = SHA-256(LE128(i a_1) | LE128(i a_2) | LE128(i a_3)),
  // digest read as a big-endian integer, mod k_i.
  for (int i = 1; i <= 3; i++) {
    uint8_t buf[48];
    for (int c = 0; c < 3; c++) {
      u128 v = a[c] * (u128)i;
      for (int byte = 0; byte < 16; byte++) buf[16 * c + byte] = (uint8_t)(v >> (8 * byte));
    }
    uint8_t d[32];
    sha256(buf, sizeof buf, d);
    K.omega_mod[i - 1][0] = 0;
    for (uint64_t kk = 1; kk <= 8; kk++) {
      uint64_t acc = 0;  // Horner over 32-bit big-endian words
      for (int w = 0; w < 8; w++) {
        uint64_t word = (uint64_t)d[4 * w] << 24 | (uint64_t)d[4 * w + 1] << 16 |
                        (uint64_t)d[4 * w + 2] << 8 | d[4 * w + 3];
        acc = ((acc << 32) + word) % kk;
      }
      K.omega_mod[i - 1][kk] = (uint8_t)acc;
    }
    K.omega[i - 1] = K.omega_mod[i - 1][p.k[i - 1]];
  }
  *out = K;
  return LC_OK;
}

void build_theta(double* table) {
  for (int w = 0; w < 8; w++) {
    const double den = pow10_rn(3 + w);
    for (int P = 0; P < 256; P++) table[w * 256 + P] = (double)P / den;
  }
}

}  // namespace lc
