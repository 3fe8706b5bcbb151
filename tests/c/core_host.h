/* Host stand-ins for the CUDA qualifiers and intrinsics that
 * paper_2401_14117_gb300/csrc/posit_core.cuh uses, so that the header's
 * integer arithmetic can be compiled and checked by g++ on a machine without
 * a GPU.  Each stand-in follows the CUDA documentation of the intrinsic:
 * funnel shifts of the 64-bit value hi:lo (wrapping the shift count modulo 32,
 * or clamping it at 32 for the ...c variants), count of leading zeros (32 for
 * 0), and round-to-nearest float conversions.  The float reciprocal and
 * reciprocal square root only seed the exact integer division and square
 * root, whose correction steps accept any estimate within their bounds. */
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#define __device__
#define __forceinline__ inline
#define __noinline__
#define __align__(x) alignas(x)

using std::max;
using std::min;

static inline int __clz(int x) { return x ? __builtin_clz((unsigned)x) : 32; }
static inline int __clzll(long long x) { return x ? __builtin_clzll((unsigned long long)x) : 64; }
static inline unsigned __funnelshift_l(unsigned lo, unsigned hi, unsigned sh) {
  sh &= 31u;
  return sh ? (hi << sh) | (lo >> (32u - sh)) : hi;
}
static inline unsigned __funnelshift_r(unsigned lo, unsigned hi, unsigned sh) {
  sh &= 31u;
  return sh ? (lo >> sh) | (hi << (32u - sh)) : lo;
}
static inline unsigned __funnelshift_lc(unsigned lo, unsigned hi, unsigned sh) {
  if (sh > 32u) sh = 32u;
  const uint64_t v = ((uint64_t)hi << 32) | lo;
  return sh == 32u ? lo : (unsigned)((v << sh) >> 32);
}
static inline unsigned __funnelshift_rc(unsigned lo, unsigned hi, unsigned sh) {
  if (sh > 32u) sh = 32u;
  const uint64_t v = ((uint64_t)hi << 32) | lo;
  return (unsigned)(v >> sh);
}
static inline long long __double_as_longlong(double d) {
  long long x;
  std::memcpy(&x, &d, 8);
  return x;
}
static inline double __longlong_as_double(long long x) {
  double d;
  std::memcpy(&d, &x, 8);
  return d;
}
static inline float __frcp_rn(float x) { return 1.0f / x; }
static inline float __frsqrt_rn(float x) { return 1.0f / std::sqrt(x); }
static inline float __uint2float_rn(unsigned x) { return (float)x; }
static inline float __ull2float_rn(unsigned long long x) { return (float)x; }
static inline float __ll2float_rn(long long x) { return (float)x; }
static inline unsigned __float2uint_rz(float x) { return (unsigned)x; }
static inline int __float2int_rz(float x) { return (int)x; }
