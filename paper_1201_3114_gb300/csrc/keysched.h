// keysched.h -- host-side key schedule of the Lorenz cipher (Sec. 3.1).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "../../include/lc.h"

namespace lc {

typedef unsigned __int128 u128;

struct HostKey {
  u128 a[3];         // Eqs. 2-4
  uint32_t L, D;     // L = floor(n/3); least D with 10^D >= 2^(8(L+1))
  double aprime[3];  // g(a_i)
  uint32_t mu[3];    // initial mu (Sec. 3.1)
  uint32_t omega[3]; // Eq. 7 with the parameters' k
  uint8_t omega_mod[3][9];  // hash(i a) mod k for every k = 1..8 (per-request k)
};

// FIPS 180-4 SHA-256.
void sha256(const uint8_t* msg, size_t len, uint8_t out[32]);

// Round-to-nearest-even conversion of a 128-bit unsigned integer.
double u128_to_double(u128 v);

// Correctly rounded binary64 value of 10^e, 0 <= e <= 38.
double pow10_rn(int e);

// Eqs. 2-7 for a password of 1..32 bytes.  LC_ERR_PASSWORD otherwise.
lc_status key_schedule(const lc_params& p, const uint8_t* pw, size_t n, HostKey* out);

// Theta[w * 256 + P] = RN(P / 10^(3 + w)) for w < 8 (Sec. 3.2 Step 2).
void build_theta(double* table);

// Check every field of a parameter set against the documented ranges.
bool params_valid(const lc_params& p);

}  // namespace lc
