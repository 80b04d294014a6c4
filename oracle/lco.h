/*
 * lco.h -- CPU oracle for the Lorenz-attractor chaotic cipher of
 * Marco, Martinez & Bruno, "Fast, parallel and secure cryptography algorithm
 * using Lorenz's attractor" (arXiv 1201.3114).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct
 * definition that the CUDA library is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline / reference arm may load it.
 * The product library shares no code with it and never calls it.
 *
 * Arithmetic: IEEE-754 binary64, round-to-nearest-even, one rounding per
 * operation, no contraction (built with -O2 -ffp-contract=off).  Every
 * function cites the passage of the paper it follows.
 *
 * Pins (see the tests under tests/test_oracle_*.py):
 *   lco_euler_step      fixed point, invariant z-axis, first-order
 *                       convergence to the Lorenz flow (Sec. 3.1, Eq. 1)
 *   lco_key_schedule    hand-derived worked values of Eqs. 2-4; exact
 *                       integer/Python-float re-derivation of a', D, mu;
 *                       SHA-256 against hashlib (Sec. 3.1, Eqs. 5-7)
 *   lco_rbyte           hand-derived integer values (Eq. 8)
 *   lco_encode/decode   the Caesar cipher of Sec. 1, exhaustive D(E(x)) = x
 *   lco_step_byte       frozen-dynamics special cases that reduce to a Caesar
 *                       key stream (Sec. 1); each sub-step of Steps 1-3
 *                       (Sec. 3.2) against closed forms of one Euler step on
 *                       the z-axis and at (0, y, z): the kick target r[mu_3],
 *                       Theta, kick before F, the mu / alpha / Omega order,
 *                       r += a' last, decryption kicking with the recovered P
 *   lco_block_begin     the start point (Eq. 5 + part offset) and the warm-up
 *                       length as z0 (1 - beta dt)^n_warm on the z-axis
 *   lco_encrypt/decrypt round trip, tamper rejection, parallel == sequential
 *                       where the split is trivial (Sec. 2, Sec. 5)
 * Copies of lco.c with planted misreadings (tests/test_oracle_mutants.py)
 * must each fail one of these pins.
 * The ciphertext values of a full chaotic run are not printed in the paper:
 * for those the oracle is the definition ("parity unpinned" against printed
 * values; pinned only through the invariants above).
 */
#ifndef LCO_H
#define LCO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  LCO_OK = 0,
  LCO_ERR_ARG = 1,
  LCO_ERR_PASSWORD = 2,
  LCO_ERR_LENGTH = 3,
  LCO_ERR_INTEGRITY = 4
};

enum { LCO_ENCRYPT = 0, LCO_DECRYPT = 1 };
enum { LCO_PARALLEL = 0, LCO_SEQUENTIAL = 1 };

/* Method constants.  Sec. 3.1 gives sigma, rho, beta, the range of dt, the
 * ranges of lambda and k, and n_it; the values the paper leaves open are
 * fixed by the reading documented in lco_params_v1(). */
typedef struct {
  double sigma, rho, beta; /* Lorenz parameters (Sec. 3.1) */
  double dt;               /* Euler step, 0 < dt <= 0.027 (Sec. 3.1) */
  uint32_t n_warm;         /* Euler steps before the first byte (n_it) */
  uint32_t steps_per_byte; /* applications of F per byte (Sec. 2: one) */
  double lambda[3];        /* offset of the starting point (Eq. 5) */
  uint32_t k[3];           /* Omega_i ranges over [0, k_i) (Eq. 7) */
  uint32_t block_len;      /* bytes per parallel part (Sec. 5) */
  uint32_t tag_len;        /* integrity bytes per part (Sec. 2) */
  double eta;              /* per-part offset of the starting point */
  uint32_t omega_alpha_shift; /* Step 3's alpha index [(i+2) mod 3]+1 read with
                                 1-based i (0: alpha_i) or 0-based i (1: a
                                 cyclic shift); reading R14 */
  uint32_t reserved;
} lco_params;

/* Key material derived from the password (Sec. 3.1, Eqs. 2-7). */
typedef struct {
  uint64_t a_lo[3], a_hi[3]; /* a_i as 128-bit unsigned integers */
  uint32_t L, D;             /* L = floor(n_pi/3); 10^D >= 2^(8(L+1)) */
  double aprime[3];          /* a'_i = g(a_i) */
  uint32_t mu[3];            /* initial mu_i in {0,1,2} */
  uint32_t omega[3];         /* initial Omega_i in [0, k_i) */
} lco_key;

/* Per-trajectory state (Sec. 3.2). */
typedef struct {
  double r[3];
  double alpha[3];
  uint32_t mu[3];
  uint32_t omega[3];
} lco_state;

/* Optional run statistics: the chaos gate, and the digit statistics of the
 * trajectory coordinates of Fig. 1 (Sec. 3.1).  After the Euler step(s) of
 * every byte (body and tag), each coordinate v of r is counted with
 *   int_part[c][trunc(v) + 64]  (trunc toward zero, clamped to 0..127),
 *   digits[c][j][floor(RN(|v| 10^(2j+2))) mod 100]  for the decimal digit
 *                               pairs 1-2, 3-4 and 5-6 (j = 0, 1, 2),
 * or, when |v| >= 2^31 or v is NaN, in out_of_range[c] only. */
typedef struct {
  double max_abs_r;       /* max |r_j| seen after any Euler step */
  uint64_t r1_hist[256];  /* histogram of R_nu(alpha_1, Omega_1) */
  uint64_t steps;         /* bytes processed */
  uint64_t int_part[3][128];
  uint64_t digits[3][3][100];
  uint64_t out_of_range[3];
} lco_stats;

void lco_params_v1(lco_params* p);
int lco_params_check(const lco_params* p);

/* FIPS 180-4 SHA-256, the "hash such as MD5 or SHA" of Eq. 7. */
void lco_sha256(const uint8_t* msg, size_t len, uint8_t out[32]);

/* Eqs. 2-7.  Password length 1..32 bytes, else LCO_ERR_PASSWORD. */
int lco_key_schedule(const lco_params* p, const uint8_t* pw, size_t pw_len,
                     lco_key* key);

/* Eq. 1 read as forward Euler of the Lorenz system. */
void lco_euler_step(const lco_params* p, double r[3]);

/* floor(v) saturated to int64, NaN -> 0. */
int64_t lco_sat_floor_i64(double v);

/* Eq. 8: byte Omega of floor(alpha * 10^13) (two's complement). */
uint32_t lco_rbyte(double alpha, uint32_t omega);

/* Eqs. 9 and 10 for one byte. */
uint32_t lco_encode_byte(uint32_t x, uint32_t r1, uint32_t r2);
uint32_t lco_decode_byte(uint32_t y, uint32_t r1, uint32_t r2);

/* Start of the trajectory of part b (Eq. 5 plus the per-part offset). */
void lco_block_begin(const lco_params* p, const lco_key* key, uint64_t b,
                     lco_state* st);

/* Steps 1-3 of Sec. 3.2 for one byte x.  dir = LCO_ENCRYPT: x is P_i and
 * the return value is C_i.  dir = LCO_DECRYPT: x is C_i, the return value
 * is P_i.  stats may be NULL. */
uint32_t lco_step_byte(const lco_params* p, const lco_key* key, lco_state* st,
                       uint32_t x, int dir, lco_stats* stats);

size_t lco_nblocks(const lco_params* p, size_t n, int mode);
size_t lco_ciphertext_len(const lco_params* p, size_t n, int mode);
int lco_plaintext_len(const lco_params* p, size_t c_len, int mode, size_t* n);

/* Whole-message encryption: C has lco_ciphertext_len() bytes. */
int lco_encrypt(const lco_params* p, const uint8_t* pw, size_t pw_len,
                const uint8_t* P, size_t n, uint8_t* C, int mode);
/* Whole-message decryption: P has n bytes; on LCO_ERR_INTEGRITY P is zeroed. */
int lco_decrypt(const lco_params* p, const uint8_t* pw, size_t pw_len,
                const uint8_t* C, size_t c_len, uint8_t* P, int mode);

/* Parts [b0, b1) of a parallel-mode message of n bytes, for sampled checks
 * and for the multi-threaded CPU baseline.  P and C are the whole buffers. */
int lco_encrypt_blocks(const lco_params* p, const lco_key* key,
                       const uint8_t* P, size_t n, uint8_t* C, size_t b0,
                       size_t b1, lco_stats* stats);
/* block_ok[b - b0] receives 1 if the tag of part b verified, else 0. */
int lco_decrypt_blocks(const lco_params* p, const lco_key* key,
                       const uint8_t* C, size_t n, uint8_t* P, size_t b0,
                       size_t b1, uint8_t* block_ok);

#ifdef __cplusplus
}
#endif
#endif
