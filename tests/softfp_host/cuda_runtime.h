// Host stand-in for <cuda_runtime.h>, used only when tests compile the
// integer-path binary64 routines of csrc/softfp64.cuh with the host C++
// compiler.  It supplies the qualifiers and the handful of bit and
// conversion intrinsics that header uses, each written from its documented
// semantics (CUDA Math API, integer and type-casting intrinsics):
//
//   __funnelshift_l(lo, hi, s)  high 32 bits of (hi:lo) << (s & 31)
//   __funnelshift_r(lo, hi, s)  low 32 bits of (hi:lo) >> (s & 31)
//   __clz(x)                    leading zero bits of a 32-bit word (32 for 0)
//   __dadd_rn, __dmul_rn        binary64 add / multiply, round to nearest even
//   __double2ll_rd              round toward -inf, then to int64 with
//                               saturation, NaN -> 0 (cvt.rmi.s64.f64)
//
// The binary64 operations run on the host's IEEE-754 unit, so the routines'
// hardware fallbacks become host operations.  Every call of one is counted,
// which lets a test report how many of its cases took the integer path.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#define __device__
#define __host__
#define __forceinline__ inline __attribute__((always_inline))
#define __noinline__ __attribute__((noinline))

namespace sfp_host {
inline thread_local uint64_t hw_calls = 0;
}

static inline long long __double_as_longlong(double x) {
  long long r;
  memcpy(&r, &x, sizeof r);
  return r;
}
static inline double __longlong_as_double(long long b) {
  double r;
  memcpy(&r, &b, sizeof r);
  return r;
}
static inline int __double2loint(double x) { return (int)(uint32_t)(uint64_t)__double_as_longlong(x); }
static inline int __double2hiint(double x) { return (int)(uint32_t)((uint64_t)__double_as_longlong(x) >> 32); }
static inline double __hiloint2double(int hi, int lo) {
  return __longlong_as_double((long long)(((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo));
}

static inline unsigned __funnelshift_l(unsigned lo, unsigned hi, unsigned s) {
  const uint64_t v = ((uint64_t)hi << 32) | lo;
  return (unsigned)((v << (s & 31u)) >> 32);
}
static inline unsigned __funnelshift_r(unsigned lo, unsigned hi, unsigned s) {
  const uint64_t v = ((uint64_t)hi << 32) | lo;
  return (unsigned)(v >> (s & 31u));
}
static inline int __clz(int x) {
  uint32_t v = (uint32_t)x;
  int n = 0;
  if (v == 0) return 32;
  while (!(v & 0x80000000u)) {
    v <<= 1;
    n++;
  }
  return n;
}

static inline uint32_t max(uint32_t a, uint32_t b) { return a > b ? a : b; }
static inline uint32_t min(uint32_t a, uint32_t b) { return a < b ? a : b; }

static inline double __dadd_rn(double a, double b) {
  sfp_host::hw_calls++;
  return a + b;
}
static inline double __dmul_rn(double a, double b) {
  sfp_host::hw_calls++;
  return a * b;
}
static inline long long __double2ll_rd(double x) {
  sfp_host::hw_calls++;
  if (isnan(x)) return 0;
  const double f = floor(x);
  if (f >= 9223372036854775808.0) return INT64_MAX;
  if (f < -9223372036854775808.0) return INT64_MIN;
  return (long long)f;
}
