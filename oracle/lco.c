/*
 * lco.c -- CPU oracle for the Lorenz-attractor chaotic cipher (arXiv 1201.3114).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline arm; never by the product library.
 *
 * Plain C99 (plus unsigned __int128), IEEE-754 binary64 round-to-nearest-even,
 * built with -O2 -ffp-contract=off so that every written operation is one
 * rounding.  Each function names the passage of the paper it restates.
 * Where the paper is silent, ambiguous or garbled, the reading taken is
 * stated next to the code as a numbered reading (R1..R22).
 */
#include "lco.h"

#include <math.h>
#include <string.h>

typedef unsigned __int128 u128;

/* Correctly rounded binary64 values of 10^e, written as decimal literals
 * (the compiler rounds each literal to nearest).  Exact up to 10^22. */
static const double TEN[28] = {
    1e0,  1e1,  1e2,  1e3,  1e4,  1e5,  1e6,  1e7,  1e8,  1e9,
    1e10, 1e11, 1e12, 1e13, 1e14, 1e15, 1e16, 1e17, 1e18, 1e19,
    1e20, 1e21, 1e22, 1e23, 1e24, 1e25, 1e26, 1e27};

/* nu = floor(log10 2^(xi-6)) with xi = 52 (Sec. 3.1): log10 2^46 = 13.85. */
#define LCO_NU 13

/* ---------------------------------------------------------------------- */
/* Parameters                                                              */
/* ---------------------------------------------------------------------- */

/* Sec. 3.1: sigma = 10, rho = 28, beta = 8/3 (rounded once, reading R3),
 * 0 < dt <= 0.027 (reading R2: dt = 0.01), n_it = 3000 taken as the number
 * of Euler steps before the first byte (reading R4), one application of F
 * per byte as in r_i = F[r_{i-1} + M(P_i)] of Sec. 2.  lambda is only given
 * as ranges (Eq. 5); reading R10 takes (1, 1, 20), inside them.  k_i must
 * satisfy 2 < k_i <= floor((52-14)/8) = 4 (Eq. 7); reading R11 takes 4.
 * The parallel split of Sec. 5 uses fixed 4096-byte parts (reading R18) and
 * each part carries an 8-byte integrity tag (reading R19). */
void lco_params_v1(lco_params* p) {
  p->sigma = 10.0;
  p->rho = 28.0;
  p->beta = 8.0 / 3.0;
  p->dt = 0.01;
  p->n_warm = 3000;
  p->steps_per_byte = 1;
  p->lambda[0] = 1.0;
  p->lambda[1] = 1.0;
  p->lambda[2] = 20.0;
  p->k[0] = 4;
  p->k[1] = 4;
  p->k[2] = 4;
  p->block_len = 4096;
  p->tag_len = 8;
  p->eta = 0x1p-24;
  p->omega_alpha_shift = 0; /* reading R14 */
  p->reserved = 0;
}

int lco_params_check(const lco_params* p) {
  int i;
  if (p->block_len == 0 || p->tag_len == 0 || p->tag_len > 8) return LCO_ERR_ARG;
  if (p->omega_alpha_shift > 1) return LCO_ERR_ARG;
  for (i = 0; i < 3; i++)
    if (p->k[i] < 1 || p->k[i] > 8) return LCO_ERR_ARG;
  /* Theta divides by 10^(3 + Omega_3): Omega_3 <= 7 keeps it in TEN[]. */
  return LCO_OK;
}

/* ---------------------------------------------------------------------- */
/* SHA-256 (FIPS 180-4), the hash of Eq. 7 (reading R12)                   */
/* ---------------------------------------------------------------------- */

static const uint32_t SHA_K[64] = {
    0x428a2f98u, 0x71374491u, 0xb5c0fbcfu, 0xe9b5dba5u, 0x3956c25bu, 0x59f111f1u,
    0x923f82a4u, 0xab1c5ed5u, 0xd807aa98u, 0x12835b01u, 0x243185beu, 0x550c7dc3u,
    0x72be5d74u, 0x80deb1feu, 0x9bdc06a7u, 0xc19bf174u, 0xe49b69c1u, 0xefbe4786u,
    0x0fc19dc6u, 0x240ca1ccu, 0x2de92c6fu, 0x4a7484aau, 0x5cb0a9dcu, 0x76f988dau,
    0x983e5152u, 0xa831c66du, 0xb00327c8u, 0xbf597fc7u, 0xc6e00bf3u, 0xd5a79147u,
    0x06ca6351u, 0x14292967u, 0x27b70a85u, 0x2e1b2138u, 0x4d2c6dfcu, 0x53380d13u,
    0x650a7354u, 0x766a0abbu, 0x81c2c92eu, 0x92722c85u, 0xa2bfe8a1u, 0xa81a664bu,
    0xc24b8b70u, 0xc76c51a3u, 0xd192e819u, 0xd6990624u, 0xf40e3585u, 0x106aa070u,
    0x19a4c116u, 0x1e376c08u, 0x2748774cu, 0x34b0bcb5u, 0x391c0cb3u, 0x4ed8aa4au,
    0x5b9cca4fu, 0x682e6ff3u, 0x748f82eeu, 0x78a5636fu, 0x84c87814u, 0x8cc70208u,
    0x90befffau, 0xa4506cebu, 0xbef9a3f7u, 0xc67178f2u};

static uint32_t rotr32(uint32_t x, int n) { return (x >> n) | (x << (32 - n)); }

static void sha256_block(uint32_t h[8], const uint8_t blk[64]) {
  uint32_t w[64], a, b, c, d, e, f, g, hh, t1, t2, s0, s1;
  int t;
  for (t = 0; t < 16; t++)
    w[t] = ((uint32_t)blk[4 * t] << 24) | ((uint32_t)blk[4 * t + 1] << 16) |
           ((uint32_t)blk[4 * t + 2] << 8) | (uint32_t)blk[4 * t + 3];
  for (t = 16; t < 64; t++) {
    s0 = rotr32(w[t - 15], 7) ^ rotr32(w[t - 15], 18) ^ (w[t - 15] >> 3);
    s1 = rotr32(w[t - 2], 17) ^ rotr32(w[t - 2], 19) ^ (w[t - 2] >> 10);
    w[t] = w[t - 16] + s0 + w[t - 7] + s1;
  }
  a = h[0]; b = h[1]; c = h[2]; d = h[3];
  e = h[4]; f = h[5]; g = h[6]; hh = h[7];
  for (t = 0; t < 64; t++) {
    s1 = rotr32(e, 6) ^ rotr32(e, 11) ^ rotr32(e, 25);
    t1 = hh + s1 + ((e & f) ^ (~e & g)) + SHA_K[t] + w[t];
    s0 = rotr32(a, 2) ^ rotr32(a, 13) ^ rotr32(a, 22);
    t2 = s0 + ((a & b) ^ (a & c) ^ (b & c));
    hh = g; g = f; f = e; e = d + t1;
    d = c; c = b; b = a; a = t1 + t2;
  }
  h[0] += a; h[1] += b; h[2] += c; h[3] += d;
  h[4] += e; h[5] += f; h[6] += g; h[7] += hh;
}

void lco_sha256(const uint8_t* msg, size_t len, uint8_t out[32]) {
  uint32_t h[8] = {0x6a09e667u, 0xbb67ae85u, 0x3c6ef372u, 0xa54ff53au,
                   0x510e527fu, 0x9b05688cu, 0x1f83d9abu, 0x5be0cd19u};
  uint8_t blk[64];
  size_t off = 0, rem;
  uint64_t bits = (uint64_t)len * 8u;
  int i;
  while (len - off >= 64) {
    sha256_block(h, msg + off);
    off += 64;
  }
  rem = len - off;
  memset(blk, 0, sizeof blk);
  if (rem) memcpy(blk, msg + off, rem);
  blk[rem] = 0x80;
  if (rem >= 56) {
    sha256_block(h, blk);
    memset(blk, 0, sizeof blk);
  }
  for (i = 0; i < 8; i++) blk[63 - i] = (uint8_t)(bits >> (8 * i));
  sha256_block(h, blk);
  for (i = 0; i < 8; i++) {
    out[4 * i] = (uint8_t)(h[i] >> 24);
    out[4 * i + 1] = (uint8_t)(h[i] >> 16);
    out[4 * i + 2] = (uint8_t)(h[i] >> 8);
    out[4 * i + 3] = (uint8_t)h[i];
  }
}

/* ---------------------------------------------------------------------- */
/* Key schedule, Sec. 3.1                                                  */
/* ---------------------------------------------------------------------- */

/* pi_i with the paper's 1-based index. */
static u128 PI(const uint8_t* pw, size_t i) { return (u128)pw[i - 1]; }

static uint32_t mod3_u128(u128 v) { return (uint32_t)(v % 3u); }

/* Big-endian 256-bit integer modulo m (m <= 8), by Horner over the bytes. */
static uint32_t be256_mod(const uint8_t d[32], uint32_t m) {
  uint32_t r = 0;
  int i;
  for (i = 0; i < 32; i++) r = (r * 256u + d[i]) % m;
  return r;
}

static void le128(u128 v, uint8_t* out) {
  int i;
  for (i = 0; i < 16; i++) out[i] = (uint8_t)(v >> (8 * i));
}

int lco_key_schedule(const lco_params* p, const uint8_t* pw, size_t n,
                     lco_key* K) {
  size_t L, q, i;
  u128 a[3] = {0, 0, 0}, lim, p10;
  uint32_t D, mu_sum;
  int j;

  if (pw == NULL || n < 1 || n > 32) return LCO_ERR_PASSWORD; /* reading R8 */
  L = n / 3;
  q = n % 3;

  /* Eq. 2 */
  if (q == 0) {
    for (i = 1; i <= L; i++) a[0] += PI(pw, i) << (8 * (i - 1));
  } else {
    for (i = 1; i <= L; i++) a[0] += PI(pw, i) << (8 * i);
    a[0] += PI(pw, 3 * L + 1);
  }
  /* Eq. 3 */
  if (q != 2) {
    for (i = L + 1; i <= 2 * L; i++) a[1] += PI(pw, i) << (8 * (i - L - 1));
  } else {
    for (i = L + 1; i <= 2 * L; i++) a[1] += PI(pw, i) << (8 * (i - L));
    a[1] += PI(pw, 3 * L + 2);
  }
  /* Eq. 4 */
  for (i = 2 * L + 1; i <= 3 * L; i++) a[2] += PI(pw, i) << (8 * (i - 2 * L - 1));

  /* g(x) = x / 10^ceil(log10 2^(8(L+1))) (reading R5: decimal log).
   * D is the least integer with 10^D >= 2^(8(L+1)), found exactly. */
  lim = (u128)1 << (8 * (L + 1));
  D = 0;
  p10 = 1;
  while (p10 < lim) {
    p10 *= 10u;
    D++;
  }

  for (j = 0; j < 3; j++) {
    K->a_lo[j] = (uint64_t)a[j];
    K->a_hi[j] = (uint64_t)(a[j] >> 64);
    /* one rounding for the integer, one for the division (reading R9) */
    K->aprime[j] = (double)a[j] / TEN[D];
  }
  K->L = (uint32_t)L;
  K->D = D;

  /* mu from a mod 3 (Sec. 3.1), reduced first so the products fit. */
  mu_sum = mod3_u128(a[0]) + mod3_u128(a[1]) + mod3_u128(a[2]);
  K->mu[0] = mu_sum % 3u;
  K->mu[1] = (mod3_u128(a[0]) * mod3_u128(a[1]) + mod3_u128(a[2])) % 3u;
  K->mu[2] = (mod3_u128(a[0]) + mod3_u128(a[1]) * mod3_u128(a[2])) % 3u;

  /* Eq. 7: Omega_i = hash(i a) mod k_i.  Reading R12: SHA-256 of the three
   * products as 16-byte little-endian integers, digest read big-endian. */
  for (j = 0; j < 3; j++) {
    uint8_t msg[48], dig[32];
    int c;
    for (c = 0; c < 3; c++) le128((u128)(j + 1) * a[c], msg + 16 * c);
    lco_sha256(msg, sizeof msg, dig);
    K->omega[j] = be256_mod(dig, p->k[j]);
  }
  return LCO_OK;
}

/* ---------------------------------------------------------------------- */
/* Dynamics, Sec. 3.1 Eq. 1                                                */
/* ---------------------------------------------------------------------- */

/* Reading R1: Eq. 1 as printed multiplies the whole right-hand side by dt,
 * which makes the origin attracting (no chaos).  The text names the Euler
 * discretisation of the Lorenz system, so this is standard forward Euler:
 *   x' = x + dt * (sigma (y - x))
 *   y' = y + dt * ((rho x - y) - x z)
 *   z' = z + dt * (x y - beta z)
 * with exactly this operation order. */
void lco_euler_step(const lco_params* p, double r[3]) {
  double x = r[0], y = r[1], z = r[2];
  double dx = p->sigma * (y - x);
  double dy = (p->rho * x - y) - x * z;
  double dz = x * y - p->beta * z;
  r[0] = x + p->dt * dx;
  r[1] = y + p->dt * dy;
  r[2] = z + p->dt * dz;
}

/* ---------------------------------------------------------------------- */
/* Byte extractor and byte map, Sec. 3.1 Eqs. 8-10                         */
/* ---------------------------------------------------------------------- */

/* floor() saturated to the int64 range; NaN maps to 0 (reading R7). */
int64_t lco_sat_floor_i64(double v) {
  if (isnan(v)) return 0;
  if (v >= 9223372036854775808.0) return INT64_MAX;
  if (v < -9223372036854775808.0) return INT64_MIN;
  return (int64_t)floor(v);
}

/* Eq. 8: R_nu(alpha, Omega) = (floor(alpha 10^nu) AND 255*2^(8 Omega)) / 2^(8 Omega)
 * with nu = 13 (reading R5), the integer held as a two's complement int64
 * (readings R6, R7). */
uint32_t lco_rbyte(double alpha, uint32_t omega) {
  double v = alpha * TEN[LCO_NU];
  uint64_t V = (uint64_t)lco_sat_floor_i64(v);
  return (uint32_t)((V >> (8u * omega)) & 255u);
}

/* Eq. 9 */
uint32_t lco_encode_byte(uint32_t x, uint32_t r1, uint32_t r2) {
  return (x + r1 + r2) % 256u;
}

/* Eq. 10: the residue is taken non-negative (Sec. 1 on the sign flip). */
uint32_t lco_decode_byte(uint32_t y, uint32_t r1, uint32_t r2) {
  int v = (int)y - (int)r1 - (int)r2;
  v %= 256;
  if (v < 0) v += 256;
  return (uint32_t)v;
}

/* ---------------------------------------------------------------------- */
/* One trajectory, Sec. 3.2 and Sec. 5                                     */
/* ---------------------------------------------------------------------- */

/* Eq. 5, r_0 = a' + lambda, plus the offset b*eta that gives each parallel
 * part its own initial condition (Sec. 5, reading R18); then n_it Euler
 * steps (reading R4) and Eq. 6 for alpha (sampled after the warm-up,
 * reading R17). */
void lco_block_begin(const lco_params* p, const lco_key* K, uint64_t b,
                     lco_state* st) {
  int j;
  uint32_t s;
  for (j = 0; j < 3; j++)
    st->r[j] = (K->aprime[j] + p->lambda[j]) + (double)b * p->eta;
  for (s = 0; s < p->n_warm; s++) lco_euler_step(p, st->r);
  for (j = 0; j < 3; j++) {
    st->mu[j] = K->mu[j];
    st->omega[j] = K->omega[j];
    st->alpha[j] = st->r[st->mu[j]];
  }
}

/* Fig. 1 (Sec. 3.1): the integer part and the decimal digit pairs 1-2, 3-4
 * and 5-6 of a coordinate, read from its sign-magnitude decimal expansion:
 * trunc(v), and floor(|v| 10^(2j+2)) mod 100 with the product rounded once. */
static void count_digits(lco_stats* stats, int c, double v) {
  static const double scale[3] = {1e2, 1e4, 1e6};
  double a = fabs(v);
  int j, ip;
  if (!(a < 2147483648.0)) { /* also NaN */
    stats->out_of_range[c]++;
    return;
  }
  ip = (int)v; /* toward zero */
  ip += 64;
  if (ip < 0) ip = 0;
  if (ip > 127) ip = 127;
  stats->int_part[c][ip]++;
  for (j = 0; j < 3; j++) {
    uint64_t u = (uint64_t)floor(a * scale[j]);
    stats->digits[c][j][u % 100u]++;
  }
}

static void stats_r(lco_stats* stats, const double r[3]) {
  int j;
  for (j = 0; j < 3; j++) {
    double m = fabs(r[j]);
    if (isnan(m) || m > stats->max_abs_r) stats->max_abs_r = m; /* NaN sticks */
    count_digits(stats, j, r[j]);
  }
}

/* Sec. 3.2, Steps 1-3, for one byte. */
uint32_t lco_step_byte(const lco_params* p, const lco_key* K, lco_state* st,
                       uint32_t x, int dir, lco_stats* stats) {
  uint32_t r1, r2, y, P, s;
  int i;
  double theta;

  /* Step 1: Eq. 9 (encrypt) or Eq. 10 (decrypt) with alpha_1, alpha_2. */
  r1 = lco_rbyte(st->alpha[0], st->omega[0]);
  r2 = lco_rbyte(st->alpha[1], st->omega[1]);
  if (dir == LCO_ENCRYPT) {
    P = x;
    y = lco_encode_byte(x, r1, r2);
  } else {
    y = lco_decode_byte(x, r1, r2);
    P = y; /* reading R16: the recovered plaintext drives Step 2 */
  }
  if (stats) {
    stats->r1_hist[r1]++;
    stats->steps++;
  }

  /* Step 2: Theta = P_i / 10^(3 + Omega_3) is added to the component of r
   * picked by mu_3 (reading R15: the state, as in r_i = F[r_{i-1} + M(P_i)]
   * of Sec. 2), then F is applied. */
  theta = (double)P / TEN[3 + st->omega[2]];
  st->r[st->mu[2]] = st->r[st->mu[2]] + theta;
  for (s = 0; s < p->steps_per_byte; s++) lco_euler_step(p, st->r);
  if (stats) stats_r(stats, st->r);

  /* Step 3 (reading R13 for the order):
   *   mu_i    <- (mu_i + R(alpha_i, Omega_i)) mod 3     old alpha, old Omega
   *   alpha_i <- r[mu_i]                                Eq. 6, new mu
   *   Omega_i <- (Omega_i + R(alpha_j, Omega_i)) mod k_i  new alpha, old Omega
   *            j = [(i+2) mod 3]+1: with 1-based i that is i (reading R14,
   *            the default); with 0-based i (omega_alpha_shift = 1) it is
   *            the cyclic predecessor of i
   *   r       <- r + a'                                                   */
  for (i = 0; i < 3; i++)
    st->mu[i] = (st->mu[i] + lco_rbyte(st->alpha[i], st->omega[i])) % 3u;
  for (i = 0; i < 3; i++) st->alpha[i] = st->r[st->mu[i]];
  for (i = 0; i < 3; i++)
    st->omega[i] = (st->omega[i] + lco_rbyte(st->alpha[p->omega_alpha_shift ? (i + 2) % 3 : i],
                                             st->omega[i])) % p->k[i];
  for (i = 0; i < 3; i++) st->r[i] = st->r[i] + K->aprime[i];

  return y;
}

/* ---------------------------------------------------------------------- */
/* Framing: parts, tags and lengths (Sec. 2, Sec. 5; readings R18-R21)     */
/* ---------------------------------------------------------------------- */

size_t lco_nblocks(const lco_params* p, size_t n, int mode) {
  if (mode == LCO_SEQUENTIAL || n == 0) return 1;
  return (n + p->block_len - 1) / p->block_len;
}

size_t lco_ciphertext_len(const lco_params* p, size_t n, int mode) {
  return n + (size_t)p->tag_len * lco_nblocks(p, n, mode);
}

int lco_plaintext_len(const lco_params* p, size_t c_len, int mode, size_t* n) {
  size_t m, cand;
  if (c_len < p->tag_len) return LCO_ERR_LENGTH;
  if (mode == LCO_SEQUENTIAL) {
    *n = c_len - p->tag_len;
    return LCO_OK;
  }
  /* Search the block counts near c_len / (B + T); exactly one may fit. */
  m = c_len / ((size_t)p->block_len + p->tag_len);
  for (cand = (m > 0 ? m : 1); cand <= m + 1; cand++) {
    size_t nn;
    if ((size_t)p->tag_len * cand > c_len) break;
    nn = c_len - (size_t)p->tag_len * cand;
    if (lco_nblocks(p, nn, LCO_PARALLEL) == cand) {
      *n = nn;
      return LCO_OK;
    }
  }
  return LCO_ERR_LENGTH;
}

/* The tag plaintext Q: the message length as 8 little-endian bytes. */
static uint32_t tag_plain(size_t n, uint32_t t) {
  return (uint32_t)(((uint64_t)n >> (8 * t)) & 255u);
}

int lco_encrypt_blocks(const lco_params* p, const lco_key* K, const uint8_t* P,
                       size_t n, uint8_t* C, size_t b0, size_t b1,
                       lco_stats* stats) {
  size_t b, i, lo, hi;
  uint32_t t;
  lco_state st;
  for (b = b0; b < b1; b++) {
    lco_block_begin(p, K, b, &st);
    lo = b * p->block_len;
    hi = lo + p->block_len;
    if (hi > n) hi = n;
    for (i = lo; i < hi; i++)
      C[i] = (uint8_t)lco_step_byte(p, K, &st, P[i], LCO_ENCRYPT, stats);
    for (t = 0; t < p->tag_len; t++)
      C[n + b * p->tag_len + t] =
          (uint8_t)lco_step_byte(p, K, &st, tag_plain(n, t), LCO_ENCRYPT, stats);
  }
  return LCO_OK;
}

int lco_decrypt_blocks(const lco_params* p, const lco_key* K, const uint8_t* C,
                       size_t n, uint8_t* P, size_t b0, size_t b1,
                       uint8_t* block_ok) {
  size_t b, i, lo, hi;
  uint32_t t;
  lco_state st;
  for (b = b0; b < b1; b++) {
    int ok = 1;
    lco_block_begin(p, K, b, &st);
    lo = b * p->block_len;
    hi = lo + p->block_len;
    if (hi > n) hi = n;
    for (i = lo; i < hi; i++)
      P[i] = (uint8_t)lco_step_byte(p, K, &st, C[i], LCO_DECRYPT, NULL);
    for (t = 0; t < p->tag_len; t++) {
      uint32_t q = lco_step_byte(p, K, &st, C[n + b * p->tag_len + t],
                                 LCO_DECRYPT, NULL);
      if (q != tag_plain(n, t)) ok = 0;
    }
    block_ok[b - b0] = (uint8_t)ok;
  }
  return LCO_OK;
}

int lco_encrypt(const lco_params* p, const uint8_t* pw, size_t pw_len,
                const uint8_t* P, size_t n, uint8_t* C, int mode) {
  lco_key K;
  lco_state st;
  size_t i;
  uint32_t t;
  int rc = lco_params_check(p);
  if (rc) return rc;
  rc = lco_key_schedule(p, pw, pw_len, &K);
  if (rc) return rc;
  if (mode == LCO_PARALLEL)
    return lco_encrypt_blocks(p, &K, P, n, C, 0, lco_nblocks(p, n, mode), NULL);
  /* Sequential (strong) version: one trajectory over the whole message. */
  lco_block_begin(p, &K, 0, &st);
  for (i = 0; i < n; i++)
    C[i] = (uint8_t)lco_step_byte(p, &K, &st, P[i], LCO_ENCRYPT, NULL);
  for (t = 0; t < p->tag_len; t++)
    C[n + t] = (uint8_t)lco_step_byte(p, &K, &st, tag_plain(n, t), LCO_ENCRYPT, NULL);
  return LCO_OK;
}

int lco_decrypt(const lco_params* p, const uint8_t* pw, size_t pw_len,
                const uint8_t* C, size_t c_len, uint8_t* P, int mode) {
  lco_key K;
  lco_state st;
  size_t n, i, b, nb;
  uint32_t t;
  int ok = 1;
  int rc = lco_params_check(p);
  if (rc) return rc;
  rc = lco_plaintext_len(p, c_len, mode, &n);
  if (rc) return rc;
  rc = lco_key_schedule(p, pw, pw_len, &K);
  if (rc) return rc;
  if (mode == LCO_PARALLEL) {
    nb = lco_nblocks(p, n, mode);
    for (b = 0; b < nb; b++) {
      uint8_t bok = 0;
      lco_decrypt_blocks(p, &K, C, n, P, b, b + 1, &bok);
      if (!bok) ok = 0;
    }
  } else {
    lco_block_begin(p, &K, 0, &st);
    for (i = 0; i < n; i++)
      P[i] = (uint8_t)lco_step_byte(p, &K, &st, C[i], LCO_DECRYPT, NULL);
    for (t = 0; t < p->tag_len; t++)
      if (lco_step_byte(p, &K, &st, C[n + t], LCO_DECRYPT, NULL) != tag_plain(n, t))
        ok = 0;
  }
  if (!ok) {
    if (n) memset(P, 0, n); /* fail closed */
    return LCO_ERR_INTEGRITY;
  }
  return LCO_OK;
}
