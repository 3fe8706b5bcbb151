// posit_core.cuh -- Posit(32,2) scalar arithmetic for sm_103a, integer only.
//
// Format (Sec. 2, Eq. 1): x = (-1)^s * 16^k * 2^e * 1.f.  A word is decoded
// once into a "pz" pair and all arithmetic runs on decoded values:
//
//   pz.s  scale S = 4k + e (2^S <= |x| < 2^(S+1)); zero uses PZ_SZERO,
//         NaR uses PZ_SNAR (both far outside the +-120 range of real values)
//   pz.m  sign in bit 31; magnitude 1.f with the hidden one at bit 30 and the
//         fraction below it (at most 27 fraction bits, so bits 2..0 are 0)
//
// Every multiply and every add is rounded to Posit(32,2) at once (Sec. 2,
// pre-/post-processing: operate in an internal format, re-encode the regime,
// round with the new f_s).  Rounding rule (the paper gives none): round the
// value's posit bit string to 31 bits after the sign, to nearest, ties to the
// even pattern, saturating at minpos/maxpos.  While the regime run m is at
// most 27 (-108 <= S <= 107) both exponent bits and at least one fraction bit
// fit, the last bit of the pattern is a fraction bit, and this is ordinary
// round-to-nearest-even of the significand to f_s = 28 - m fraction bits; that
// is the fast path.  From m = 28 on the last bit of the pattern is an
// exponent bit (or a regime bit), which decides ties, so those scales use the
// bit-string encoder (pz_encode).
//
// Intermediate significands carry a "jam" bit: bit 0 is set when nonzero bits
// were shifted out below it.  Rounding never keeps more than 28 bits of a
// significand whose leading one is at bit 30, so the guard bit is at bit 2 or
// higher and the jam bit only decides "exactly half" vs "more than half".
#pragma once
#include <stdint.h>

#define PZ_SZERO (-(1 << 20))
#define PZ_SNAR (1 << 22)
#define PZ_NAR_T (1 << 21)     // s >= PZ_NAR_T: NaR
#define PZ_ZERO_T (-(1 << 19)) // s <= PZ_ZERO_T: zero (then m's magnitude is 0)
#define PZ_NAR_BITS 0x80000000u
#define PZ_ONE_BITS 0x40000000u

struct pz {
  int s;
  uint32_t m;
};

static __device__ __forceinline__ pz pz_zero() { return pz{PZ_SZERO, 0u}; }
static __device__ __forceinline__ pz pz_nar() { return pz{PZ_SNAR, 1u << 30}; }
static __device__ __forceinline__ pz pz_one() { return pz{0, 1u << 30}; }
static __device__ __forceinline__ bool pz_is_nar(pz a) { return a.s >= (PZ_SNAR >> 1); }
static __device__ __forceinline__ bool pz_is_zero(pz a) { return (a.m & 0x7FFFFFFFu) == 0u; }

// ---------------------------------------------------------------------------
// word <-> decoded
// ---------------------------------------------------------------------------

// Sec. 2, Eq. 1: sign removed by two's-complement negation, regime run length
// m from a count of leading ones/zeros, then 2 exponent bits (missing bits are
// 0), then the fraction.
static __device__ __forceinline__ pz pz_decode(uint32_t p) {
  if (p == 0u) return pz_zero();
  if (p == PZ_NAR_BITS) return pz_nar();
  uint32_t sign = p & 0x80000000u;
  uint32_t a = sign ? (0u - p) : p;
  uint32_t x = a << 1;  // the 31 bits after the sign, left-aligned
  uint32_t first = x >> 31;
  int m = first ? __clz(~x) : __clz(x);  // 1..31 (x has bit 0 clear)
  int k = first ? m - 1 : -m;
  uint32_t rest = (x << m) << 1;  // drop the run and its terminating bit
  int e = (int)(rest >> 30);
  uint32_t mag = (1u << 30) | ((rest << 2) >> 2);
  return pz{4 * k + e, sign | mag};
}

// Bit-string rounding of sign * 2^S * X / 2^30 (X: leading one at bit 30,
// bit 0 possibly a jam bit) to a Posit(32,2) word.
static __device__ __noinline__ uint32_t pz_encode(uint32_t sign, int S, uint32_t X) {
  int k = S >> 2;  // floor(S / 4)
  int e = S & 3;
  uint32_t p;
  if (k >= 30) {
    p = 0x7FFFFFFFu;  // at or beyond maxpos = 2^120
  } else if (k < -30) {
    p = 1u;  // below 2^-120: minpos (never rounds to zero)
  } else {
    int L = k >= 0 ? k + 2 : 1 - k;  // regime length with terminator, 2..31
    uint64_t reg = k >= 0 ? (((1ull << (k + 1)) - 1ull) << 1) : 1ull;
    // string: regime (L bits) | e (2 bits) | the 30 bits of X below its lead
    uint64_t str = (reg << 32) | ((uint64_t)e << 30) | (uint64_t)(X & 0x3FFFFFFFu);
    // total length L + 32; keep 31 bits, the next one is the guard bit
    p = (uint32_t)(str >> (L + 1));
    uint32_t guard = (uint32_t)(str >> L) & 1u;
    uint32_t sticky = (str & ((1ull << L) - 1ull)) != 0ull;
    if (guard && (sticky || (p & 1u))) p += 1u;
    if (p > 0x7FFFFFFFu) p = 0x7FFFFFFFu;
    if (p == 0u) p = 1u;
  }
  return sign ? (0u - p) : p;
}

// Word of an already rounded decoded value (exact, no rounding happens).  The
// pattern after the sign is the regime (k+1 ones and a zero, or -k zeros and a
// one) followed by the 2 exponent bits and 27 fraction bits, cut to 31 bits;
// the bits cut off are zero because the value is a posit.
static __device__ __forceinline__ uint32_t pz_to_bits(pz a) {
  if (pz_is_nar(a)) return PZ_NAR_BITS;
  if (pz_is_zero(a)) return 0u;
  const int k = a.s >> 2;  // -30 .. 30 for every rounded value
  const uint32_t body = ((uint32_t)(a.s & 3) << 27) | ((a.m & 0x3FFFFFFFu) >> 3);
  const uint32_t pay = k >= 0 ? ((0x7FFFFFFFu ^ (0x7FFFFFFFu >> (k + 1))) | (body >> k))
                              : ((1u << (30 + k)) | (body >> (-1 - k)));
  return (a.m >> 31) ? (0u - pay) : pay;
}

// Slow rounding for regimes of 28 or more bits (S <= -109 or S >= 108).
static __device__ __noinline__ pz pz_round_band(uint32_t sign, int S, uint32_t X) {
  return pz_decode(pz_encode(sign, S, X));
}

// Round sign * 2^S * X / 2^30 (X leading one at bit 30 with jam bit, or
// X == 0 for zero, or a NaR/zero sentinel scale) to the nearest posit, kept in
// decoded form.
static __device__ __forceinline__ pz pz_round(uint32_t sign, int S, uint32_t X) {
  int km = (S >> 2) ^ (S >> 31);  // regime run length m minus 1
  if ((unsigned)(km - 27) < (1u << 17)) return pz_round_band(sign, S, X);
  // q = number of bits below the kept ones: 30 - f_s = 2 + m (3..29); the
  // zero/NaR sentinels clamp to 30, which leaves X = 0 and X = 2^30 intact
  uint32_t q = min((uint32_t)km + 3u, 30u);
  uint32_t lsb = (X >> q) & 1u;
  uint32_t r = X + ((1u << (q - 1)) - 1u) + lsb;
  r &= ~((1u << q) - 1u);
  uint32_t c = r >> 31;  // rounding carried into the next binade
  return pz{S + (int)c, sign | (r >> c)};
}

// 32-bit a * b + c on the integer multiply-add pipe.  Written as PTX so that
// the compiler keeps the multiply (by a value it cannot see, such as a power
// of two read from a table) instead of turning it back into shifts and adds
// on the ALU pipe, which is the one the multiply-add loops are bound by.
static __device__ __forceinline__ uint32_t pz_imad(uint32_t a, uint32_t b, uint32_t c) {
#ifdef __CUDA_ARCH__
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
#else  // host compilation of this header (the arithmetic identity tests)
  return a * b + c;
#endif
}

// Rounding constants per scale, for kernels that keep a 256-entry table in
// shared memory (index S + 128).  q = 2 + m bits are dropped below the kept
// ones (lead at bit 30).  Scales whose regime has 28 or more bits, and every
// scale outside [-128, 127] (zero, saturation), are marked tie = 0 and take
// the general path.
struct __align__(16) pz_rtab {
  uint32_t keep;   // ~((1 << q) - 1)
  uint32_t hm1;    // (1 << (q - 1)) - 1
  uint32_t tie;    // 1 << (31 - q): X * tie has bit q of X (the tie-breaking lsb) at bit 31
  uint32_t carry;  // 0xC0000000: added to the result word when the rounding carries out
};

static __device__ __forceinline__ pz_rtab pz_rtab_make(uint32_t q) {
  pz_rtab e;
  e.keep = 0xFFFFFFFFu << q;
  e.hm1 = (1u << (q - 1)) - 1u;
  e.tie = 1u << (31 - q);
  e.carry = 0xC0000000u;
  return e;
}

static __device__ __forceinline__ pz_rtab pz_rtab_entry(int i) {
  int S = i - 128, k = S >> 2, m = k >= 0 ? k + 1 : -k;
  if (m >= 28) return pz_rtab{0u, 0u, 0u, 0xC0000000u};
  return pz_rtab_make(2u + (uint32_t)m);
}

// Table for values known to stay inside the fast band (see pz_round_inband),
// indexed by the low 8 bits of the scale: row i holds the constants of the
// scale (int8_t)i, and the rows of scales outside the band get q = 30.  A
// zero (significand 0) may land on any row: every row rounds 0 to 0.
static __device__ __forceinline__ pz_rtab pz_rtab_inband_entry(int i) {
  pz_rtab e = pz_rtab_entry(((i ^ 128) - 128) + 128);
  if (e.tie == 0u) e = pz_rtab_make(30u);
  return e;
}

// Round to nearest, ties to even, of sign * 2^S * X / 2^30 with the constants
// of the scale S.  The tie-breaking lsb (bit q of X) comes from a multiply;
// rf = X + hm1 + lsb reaches bit 31 only when the kept bits were all ones and
// round up to 2^31 (then r = 2^31 exactly, carry c = 1, scale S + 1, 2^30).
// The sign is put in with the mask, and the carry case is fixed by adding
// c * 0xC0000000 (mod 2^32): (2^31 ^ sign) + 0xC0000000 = sign | 2^30.
static __device__ __forceinline__ pz pz_round_apply(const pz_rtab &e, uint32_t sign, int S,
                                                    uint32_t X) {
  const uint32_t lsb = pz_imad(X, e.tie, 0u) >> 31;
  const uint32_t rf = X + e.hm1 + lsb;
  const uint32_t rs = (rf & e.keep) ^ sign;
  const uint32_t c = rf >> 31;
  return pz{S + (int)c, pz_imad(c, e.carry, rs)};
}

// pz_round_apply of (X0 | jam) with the jam put into the tie bit instead:
// rounding drops the part D = X mod 2^q and carries into bit q exactly when
// D > 2^(q-1), or D = 2^(q-1) and (the lsb is odd or nonzero bits lie below
// bit 0); with hm1 = 2^(q-1) - 1 that is D + hm1 + (lsb | jam) >= 2^q, the
// same carry as (D | jam) + hm1 + lsb, one logic instruction fewer.
static __device__ __forceinline__ pz pz_round_apply_jam(const pz_rtab &e, uint32_t sign, int S,
                                                        uint32_t X0, uint32_t jam) {
  const uint32_t lsb = (pz_imad(X0, e.tie, 0u) >> 31) | jam;
  const uint32_t rf = X0 + e.hm1 + lsb;
  const uint32_t rs = (rf & e.keep) ^ sign;
  const uint32_t c = rf >> 31;
  return pz{S + (int)c, pz_imad(c, e.carry, rs)};
}

// pz_round_tab without the test for the regimes of 28 or more bits: only for
// values whose scale is in [-108, 107] or that are zero (significand 0), with
// the table of pz_rtab_inband_entry.
static __device__ __forceinline__ pz pz_round_inband(const pz_rtab *tab, uint32_t sign, int S,
                                                     uint32_t X) {
  return pz_round_apply(tab[S & 255], sign, S, X);
}

// pz_round with the per-scale constants read from the table.
static __device__ __forceinline__ pz pz_round_tab(const pz_rtab *tab, uint32_t sign, int S,
                                                  uint32_t X) {
  const pz_rtab e = tab[min((unsigned)(S + 128), 255u)];
  if (e.tie == 0u) return pz_round(sign, S, X);
  return pz_round_apply(e, sign, S, X);
}

// ---------------------------------------------------------------------------
// arithmetic
// ---------------------------------------------------------------------------

static __device__ __forceinline__ pz pz_neg(pz a) {
  if (pz_is_nar(a) || pz_is_zero(a)) return a;
  return pz{a.s, a.m ^ 0x80000000u};
}

// a (x) b, one rounding, for operands that are not NaR (zero is fine: its
// magnitude 0 gives a zero product whose scale stays far below real ones).
// The 28x28-bit significand product is exact in 64 bits; its leading one
// lands at bit 61 or 62.
// The unrounded product: sign, scale, the significand X0 (lead at bit 30) and
// the jam (1 when nonzero bits lie below X0's bit 0); pz_mul_exact ORs the
// jam into bit 0, pz_round_apply_jam takes it apart.
static __device__ __forceinline__ void pz_mul_parts(pz a, pz b, uint32_t &sign, int &S,
                                                    uint32_t &X0, uint32_t &jam) {
  uint32_t A = a.m & 0x7FFFFFFFu;  // leading one at bit 30 (or 0)
  uint32_t B = b.m << 1;           // leading one at bit 31 (or 0)
  uint64_t P = (uint64_t)A * (uint64_t)B;
  uint32_t hi = (uint32_t)(P >> 32), lo = (uint32_t)P;
  uint32_t t = hi >> 30;           // 1 if the leading one is at bit 62
  // leading one to bit 30: hi, or 2 hi = hi * (t ^ 1) + hi (a multiply-add);
  // the bits of lo only matter as the jam (the lo bit that a shift by one
  // would bring in lies below the guard bit, so it needs no special care)
  X0 = pz_imad(hi, t ^ 1u, hi);
  jam = min(lo, 1u);
  S = a.s + b.s + (int)t;
  sign = (a.m ^ b.m) & 0x80000000u;
}

static __device__ __forceinline__ void pz_mul_exact(pz a, pz b, uint32_t &sign, int &S,
                                                    uint32_t &X) {
  uint32_t X0, jam;
  pz_mul_parts(a, b, sign, S, X0, jam);
  X = X0 | jam;
}

static __device__ __forceinline__ pz pz_mul_fast(pz a, pz b) {
  uint32_t sign, X;
  int S;
  pz_mul_exact(a, b, sign, S, X);
  return pz_round(sign, S, X);
}

static __device__ __forceinline__ pz pz_mul_inband(const pz_rtab *tab, pz a, pz b) {
  uint32_t sign, X0, jam;
  int S;
  pz_mul_parts(a, b, sign, S, X0, jam);
  return pz_round_apply_jam(tab[S & 255], sign, S, X0, jam);
}

static __device__ __forceinline__ pz pz_mul_tab(const pz_rtab *tab, pz a, pz b) {
  uint32_t sign, X0, jam;
  int S;
  pz_mul_parts(a, b, sign, S, X0, jam);
  const pz_rtab e = tab[min((unsigned)(S + 128), 255u)];
  if (e.tie == 0u) return pz_round(sign, S, X0 | jam);
  return pz_round_apply_jam(e, sign, S, X0, jam);
}

// c (+) t, one rounding, for operands that are not NaR.  Sign-magnitude add
// with the smaller-scale operand shifted right by d (capped at 31) and its
// shifted-out bits jammed into bit 0.  With the larger magnitude's lead at
// bit 30, a same-sign sum stays below 2^32, and a difference is negative only
// when d = 0 (then exact).
// The unrounded sum: sign, scale and significand (lead at bit 30, jam).
static __device__ __forceinline__ void pz_add_exact(pz c, pz t, uint32_t &sign, int &Sout,
                                                    uint32_t &Xout) {
  bool sw = t.s > c.s;
  int SL = sw ? t.s : c.s;
  int SS = sw ? c.s : t.s;
  uint32_t mL = sw ? t.m : c.m;
  uint32_t mS = sw ? c.m : t.m;
  uint32_t d = min((uint32_t)(SL - SS), 31u);
  uint32_t magL = mL & 0x7FFFFFFFu;
  uint32_t magS = mS & 0x7FFFFFFFu;
  uint32_t shv = magS >> d;
  uint32_t lost = __funnelshift_r(0u, magS, d);  // magS << (32 - d), 0 if d = 0
  shv |= min(lost, 1u);
  uint32_t sub = (mL ^ mS) >> 31;
  uint32_t R = sub ? (magL - shv) : (magL + shv);
  uint32_t neg = sub & (R >> 31);  // difference went negative (d = 0 only)
  R = neg ? (0u - R) : R;
  uint32_t sgn = (mL & 0x80000000u) ^ (neg << 31);
  int lz = __clz(R);
  int sft = lz - 1;  // left shift putting the leading one at bit 30
  uint32_t X = sft >= 0 ? (R << sft) : ((R >> 1) | (R & 1u));
  int S = SL - sft;
  S = (R == 0u) ? PZ_SZERO : S;  // exact cancellation
  sign = sgn;
  Sout = S;
  Xout = X;
}

static __device__ __forceinline__ pz pz_add_fast(pz c, pz t) {
  uint32_t sign, X;
  int S;
  pz_add_exact(c, t, sign, S, X);
  return pz_round(sign, S, X);
}

// Shift that brings the leading one of x to bit 31 (the count of leading
// zeros) for x != 0, and 0xFFFFFFFF for x = 0: one bfind instruction, without
// the fix-up that makes a count of leading zeros return 32 for 0.
static __device__ __forceinline__ uint32_t pz_lead_shift(uint32_t x) {
#ifdef __CUDA_ARCH__
  uint32_t d;
  asm("bfind.shiftamt.u32 %0, %1;" : "=r"(d) : "r"(x));
  return d;
#else  // host compilation of this header (the arithmetic identity tests)
  uint32_t d = 0;
  if (x == 0u) return 0xFFFFFFFFu;
  while (!(x & 0x80000000u)) { x <<= 1; ++d; }
  return d;
#endif
}

// pz_add_exact for the in-band path: clamping funnel shifts instead of
// capping the alignment at 31 (a shift of 32 or more moves every bit into the
// jam), normalisation through the form with the leading one at bit 31, and a
// zero sum (normalisation shift 0xFFFFFFFF) placed about 2^20 below the
// larger operand's scale by a multiply-add instead of a select.  Same values
// as pz_add_exact for the in-band operands; a zero keeps a significand of 0
// and a scale far below every nonzero in-band scale.
//
// BLEND picks the larger-scale operand with multiply-adds instead of selects:
// with w = 1 when t has the larger scale (else 0), mL = c.m + w (t.m - c.m)
// and mS = t.m + w (c.m - t.m), where neg1 = 0xFFFFFFFF comes from the
// caller as a value the compiler cannot see (a kernel argument), so that the
// differences stay multiply-adds on the FMA pipe and the ALU pipe, which
// bounds the multiply-add loops, is spared the selects.
template <bool BLEND>
static __device__ __forceinline__ void pz_add_exact_inband_t(pz c, pz t, uint32_t neg1,
                                                             uint32_t &sign, int &Sout,
                                                             uint32_t &Xout) {
  int SL;
  uint32_t d, mL, mS;
  if (BLEND) {
    const int dd = c.s - t.s;
    const uint32_t w = (uint32_t)dd >> 31;  // t.s > c.s
    SL = max(c.s, t.s);
    d = (uint32_t)abs(dd);
    mL = pz_imad(w, pz_imad(c.m, neg1, t.m), c.m);
    mS = pz_imad(w, pz_imad(t.m, neg1, c.m), t.m);
  } else {
    const bool sw = t.s > c.s;
    SL = sw ? t.s : c.s;
    const int SS = sw ? c.s : t.s;
    mL = sw ? t.m : c.m;
    mS = sw ? c.m : t.m;
    d = (uint32_t)(SL - SS);
  }
  uint32_t magL = mL & 0x7FFFFFFFu;
  uint32_t magS = mS & 0x7FFFFFFFu;
  uint32_t shv = __funnelshift_rc(magS, 0u, d);   // magS >> d, 0 from 32 on
  uint32_t lost = __funnelshift_rc(0u, magS, d);  // the bits shifted out
  shv |= min(lost, 1u);
  uint32_t sub = (mL ^ mS) >> 31;
  uint32_t R = sub ? (magL - shv) : (magL + shv);
  uint32_t neg = sub & (R >> 31);  // difference went negative (d = 0 only)
  R = neg ? (0u - R) : R;
  sign = (mL & 0x80000000u) ^ (neg << 31);
  const uint32_t lz = pz_lead_shift(R);
  // lead at bit 31 (R << lz; 0 for R = 0), then back to bit 30 with the bit
  // shifted out jammed (it can only be nonzero when lz = 0)
  const uint32_t Y = __funnelshift_lc(0u, R, lz);
  Xout = (Y >> 1) | (Y & 1u);
  Sout = (SL + 1 - (int)lz) + (int)(lz & 32u) * -32768;
}

static __device__ __forceinline__ void pz_add_exact_inband(pz c, pz t, uint32_t &sign, int &Sout,
                                                           uint32_t &Xout) {
  pz_add_exact_inband_t<false>(c, t, 0u, sign, Sout, Xout);
}

static __device__ __forceinline__ pz pz_add_inband(const pz_rtab *tab, pz c, pz t) {
  uint32_t sign, X;
  int S;
  pz_add_exact_inband(c, t, sign, S, X);
  return pz_round_inband(tab, sign, S, X);
}

// pz_add_inband with the operand pick by multiply-adds (neg1 = 0xFFFFFFFF).
static __device__ __forceinline__ pz pz_add_inband_blend(const pz_rtab *tab, uint32_t neg1, pz c,
                                                         pz t) {
  uint32_t sign, X;
  int S;
  pz_add_exact_inband_t<true>(c, t, neg1, sign, S, X);
  return pz_round_inband(tab, sign, S, X);
}

static __device__ __forceinline__ pz pz_add_tab(const pz_rtab *tab, pz c, pz t) {
  uint32_t sign, X;
  int S;
  pz_add_exact(c, t, sign, S, X);
  return pz_round_tab(tab, sign, S, X);
}

// c (+) t with a short dependency path, for the serial chains of the
// dot-form solves (one rounded addition per link, each waiting for the last).
// Same result as pz_add_fast for every pair of non-NaR operands.  Both
// alignment directions are formed at once, so the choice of the larger operand
// is a select after the shifts instead of before them; the three normalisations
// a sum can need when it loses at most one bit -- a carry into bit 31, none, or
// one bit of cancellation -- are formed side by side from the sum, each with
// the rounding constants of its scale (SL + 1, SL, SL - 1, computed from the
// larger scale SL while the sum is formed), and the sum's magnitude picks
// one.  The rare cases go to pz_add_fast, out of line: a difference that went
// negative or cancelled more than one bit (zero included), and a larger scale
// outside [-107, 106], whose neighbours may have a regime of 28 or more bits
// (zero and NaR operands have scales far outside).
struct pz_rq {
  uint32_t hm1, keep, q;
};

// pz_add_fast out of line: the rare fallback of pz_add_serial, kept out of
// the chain's straight-line code.
static __device__ __noinline__ pz pz_add_fast_call(pz c, pz t) { return pz_add_fast(c, t); }

// Rounding constants of a scale whose regime is shorter than 28 bits.
static __device__ __forceinline__ pz_rq pz_rq_of(int S) {
  const uint32_t q = (uint32_t)((S >> 2) ^ (S >> 31)) + 3u;  // 2 + regime run length
  return pz_rq{(1u << (q - 1)) - 1u, 0xFFFFFFFFu << q, q};
}

static __device__ __forceinline__ pz pz_add_serial(pz c, pz t) {
  const uint32_t magC = c.m & 0x7FFFFFFFu, magT = t.m & 0x7FFFFFFFu;
  const int dd = c.s - t.s, nd = t.s - c.s;  // a negative count clamps to 32
  const int SL = max(c.s, t.s);
  const bool sw = nd > 0;  // t has the larger scale
  const bool sub = (int)(c.m ^ t.m) < 0;
  const uint32_t shT = __funnelshift_rc(magT, 0u, (uint32_t)dd) |
                       min(__funnelshift_rc(0u, magT, (uint32_t)dd), 1u);
  const uint32_t shC = __funnelshift_rc(magC, 0u, (uint32_t)nd) |
                       min(__funnelshift_rc(0u, magC, (uint32_t)nd), 1u);
  const uint32_t magL = sw ? magT : magC;
  const uint32_t sS = sw ? shC : shT;
  const uint32_t sign = (sw ? t.m : c.m) & 0x80000000u;
  const uint32_t Rs = magL - sS;
  const uint32_t R = sub ? Rs : magL + sS;
  const pz_rq kA = pz_rq_of(SL + 1), kB = pz_rq_of(SL), kC = pz_rq_of(SL - 1);
  const bool c0 = R >= 0x80000000u, c1 = R >= 0x40000000u;  // carry / no shift / one bit
  const uint32_t X = c0 ? ((R >> 1) | (R & 1u)) : (c1 ? R : R << 1);
  const uint32_t lsb = c0 ? (R >> (kA.q + 1u)) & 1u
                          : (c1 ? (R >> kB.q) & 1u : (R >> (kC.q - 1u)) & 1u);
  const uint32_t hm1 = c0 ? kA.hm1 : (c1 ? kB.hm1 : kC.hm1);
  const uint32_t keep = c0 ? kA.keep : (c1 ? kB.keep : kC.keep);
  const int S = c0 ? SL + 1 : (c1 ? SL : SL - 1);
  // a round-up that carries out of the significand gives exactly 2^(S+1)
  const uint32_t rf = X + hm1 + lsb;
  const bool cy = rf >= 0x80000000u;
  pz res{cy ? S + 1 : S, cy ? (sign | 0x40000000u) : (sign | (rf & keep))};
  const bool slow = (sub && (int)Rs < 0) || R < 0x20000000u || (unsigned)(SL + 107) > 213u;
  if (slow) res = pz_add_fast_call(c, t);
  return res;
}

// General a (x) b and c (+) t: NaR in, NaR out, and the zero / NaR scales
// are put back to their canonical values so that chains of operations never
// drift between the two ranges.
static __device__ __forceinline__ pz pz_canon(pz r, bool nar) {
  if (nar || r.s >= PZ_NAR_T) return pz_nar();
  if (r.s <= PZ_ZERO_T) return pz_zero();
  return r;
}

static __device__ __forceinline__ pz pz_mul(pz a, pz b) {
  return pz_canon(pz_mul_fast(a, b), pz_is_nar(a) || pz_is_nar(b));
}

static __device__ __forceinline__ pz pz_add(pz c, pz t) {
  return pz_canon(pz_add_fast(c, t), pz_is_nar(c) || pz_is_nar(t));
}

static __device__ __forceinline__ pz pz_sub(pz c, pz t) { return pz_add(c, pz_neg(t)); }

// floor(A * 2^31 / B) for significands A, B in [2^30, 2^31), and whether the
// quotient is inexact.  The estimate comes from the correctly rounded float
// reciprocal of B (relative error below 2^-22, so within 2^10 of the
// quotient); one Newton-Raphson correction from the exact 64-bit remainder
// brings it within 1; a final adjustment makes 0 <= remainder < B.
static __device__ __forceinline__ uint32_t pz_sig_div(uint32_t A, uint32_t B, uint32_t &inexact) {
  const uint64_t N = (uint64_t)A << 31;
  const float rb = __frcp_rn(__uint2float_rn(B));
  const float qf = fminf(__uint2float_rn(A) * rb * 2147483648.0f, 4294967040.0f);
  uint32_t q = __float2uint_rz(qf);
  int64_t R = (int64_t)(N - (uint64_t)q * B);
  q += (uint32_t)__float2int_rz(__ll2float_rn(R) * rb);
  R = (int64_t)(N - (uint64_t)q * B);
  for (int i = 0; i < 4 && R < 0; ++i) { q -= 1u; R += B; }
  for (int i = 0; i < 4 && R >= (int64_t)B; ++i) { q += 1u; R -= B; }
  inexact = R != 0;
  return q;
}

// floor(sqrt(N)) for N in [2^62, 2^64), and whether the root is inexact: an
// estimate from the correctly rounded float reciprocal square root, one
// Newton-Raphson correction from the exact 64-bit residual N - r^2, and a
// final adjustment making 0 <= N - r^2 <= 2 r.
static __device__ __forceinline__ uint32_t pz_sig_sqrt(uint64_t N, uint32_t &inexact) {
  const float nf = __ull2float_rn(N);
  const float y = __frsqrt_rn(nf);
  uint32_t r = __float2uint_rz(fminf(nf * y, 4294967040.0f));
  int64_t e = (int64_t)(N - (uint64_t)r * r);
  r += (uint32_t)__float2int_rz(__ll2float_rn(e) * y * 0.5f);
  e = (int64_t)(N - (uint64_t)r * r);
  for (int i = 0; i < 4 && e < 0; ++i) { r -= 1u; e += 2 * (int64_t)r + 1; }
  for (int i = 0; i < 4 && e > 2 * (int64_t)r; ++i) { e -= 2 * (int64_t)r + 1; r += 1u; }
  inexact = e != 0;
  return r;
}

// a (/) b, one rounding: 32 quotient bits of the significands plus the
// inexact (jam) bit.  pz_div_inline for straight-line code that overlaps the
// division with other work; pz_div keeps it out of line elsewhere.
static __device__ __forceinline__ pz pz_div_inline(pz a, pz b) {
  if (pz_is_nar(a) || pz_is_nar(b) || pz_is_zero(b)) return pz_nar();
  if (pz_is_zero(a)) return pz_zero();
  uint32_t A = a.m & 0x7FFFFFFFu, B = b.m & 0x7FFFFFFFu;  // both in [2^30, 2^31)
  uint32_t jam;
  const uint32_t q = pz_sig_div(A, B, jam);  // floor(A * 2^31 / B) in (2^30, 2^32)
  int S = a.s - b.s;
  uint32_t X;
  if (q >> 31) {
    X = (q >> 1) | (q & 1u) | jam;
  } else {
    X = q | jam;
    S -= 1;
  }
  return pz_round((a.m ^ b.m) & 0x80000000u, S, X);
}

static __device__ __noinline__ pz pz_div(pz a, pz b) { return pz_div_inline(a, b); }

// sqrt(a), one rounding: the integer square root of the significand scaled
// to 64 bits, plus the inexact (jam) bit.
static __device__ __noinline__ pz pz_sqrt(pz a) {
  if (pz_is_nar(a) || (a.m >> 31)) return pz_nar();
  if (pz_is_zero(a)) return pz_zero();
  uint32_t mag = a.m & 0x7FFFFFFFu;
  int S = a.s;
  uint64_t N;
  if (S & 1) {
    N = (uint64_t)mag << 33;  // value = N * 2^(S - 1 - 62); N in [2^63, 2^64)
    S -= 1;
  } else {
    N = (uint64_t)mag << 32;  // value = N * 2^(S - 62);     N in [2^62, 2^63)
  }
  uint32_t jam;
  const uint32_t r32 = pz_sig_sqrt(N, jam);  // floor(sqrt(N)) in [2^31, 2^32)
  // sqrt(value) = r * 2^((S - 62) / 2), r in [2^31, 2^32): lead at bit 31
  uint32_t X = (r32 >> 1) | (r32 & 1u) | jam;
  return pz_round(0u, S >> 1, X);
}

// ---------------------------------------------------------------------------
// double <-> posit (input conversion of the harness; same rounding rule)
// ---------------------------------------------------------------------------
static __device__ __forceinline__ uint32_t pz_from_double(double x) {
  uint64_t u = (uint64_t)__double_as_longlong(x);
  uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  int ex = (int)((u >> 52) & 0x7FF);
  uint64_t man = u & ((1ull << 52) - 1ull);
  if (ex == 0x7FF) return PZ_NAR_BITS;  // NaN, Inf
  if (ex == 0 && man == 0) return 0u;
  uint64_t sig;
  int S;
  if (ex == 0) {  // subnormal: normalise
    int lz = __clzll(man) - 11;  // leading one to bit 52
    sig = man << lz;
    S = -1022 - lz;
  } else {
    sig = man | (1ull << 52);
    S = ex - 1023;
  }
  // leading one at bit 52 -> bit 30; 22 bits shifted out go to the jam bit
  uint32_t X = (uint32_t)(sig >> 22) | (uint32_t)((sig & ((1ull << 22) - 1ull)) != 0ull);
  // |S| <= 1074 stays far from the zero/NaR sentinel scales; large |S|
  // takes the band path and saturates there
  return pz_to_bits(pz_round(sign, S, X));
}

static __device__ __forceinline__ double pz_to_double(uint32_t p) {
  pz a = pz_decode(p);
  if (pz_is_nar(a)) return __longlong_as_double(0x7FF8000000000000ll);
  if (pz_is_zero(a)) return 0.0;
  uint64_t sign = (uint64_t)(a.m >> 31) << 63;
  uint64_t ex = (uint64_t)(a.s + 1023) << 52;
  uint64_t man = (uint64_t)(a.m & 0x3FFFFFFFu) << 22;
  return __longlong_as_double((long long)(sign | ex | man));
}
