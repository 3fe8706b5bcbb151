// chain.cuh -- the rounded additions of a serial chain with few instructions
// per link: the dot-form triangular solves (reference trsm Left-Lower-
// Transpose order, Sec. 5.1) add one rounded product at a time to a running
// value, and each addition waits for the last, so one thread runs the whole
// chain and its speed is the latency and instruction count of one link.
//
// Chain values are kept signed: pzs{s, m} is m * 2^(s - 29) with m a signed
// 32-bit significand, |m| in [2^29, 2^30].  |m| = 2^30 (the value 2^(s+1))
// is a rounded sum that carried and is not renormalised: both forms add the
// same way, so the renormalisation is left out of the chain.  Zero is
// m = 0 with s = PZS_ZERO_S, NaR m = 0 with s = PZS_NAR_S.
//
// One link, c (+) t (pzs_link), for operands whose larger scale SL lies in
// [-107, 88] and whose sum does not cancel two or more leading bits:
//   * both significands are shifted right (arithmetically) to the larger
//     scale: one shift count is 0; the bits shifted out only make a sticky
//     bit st;
//   * R = the sum, exact but for st (|R| < 2^31: one operand at most is the
//     carried 2^30);
//   * the result's leading bit is at 30 (a carry), 29, or 28 (one bit
//     cancelled); all three roundings are formed from R side by side, each
//     at the last bit its scale keeps (posit(32,2): 28 - km significant bits
//     at scale S, km = k xor (k >> 31), k = floor(S / 4)) with
//     R + (2^(p-1) - 1) + (bit p of R | st), then masked -- round to nearest
//     even with the sticky bit as the tie breaker (the A form is halved
//     after rounding, the C form rounds 2R);
//   * |R| against 2^30 and 2^29 picks one.
// The per-scale constants come from a 256-entry table indexed by SL & 255
// (shared memory: computing them costs more instructions than the link's
// other steps together).  A link whose |R| is below 2^28 (two or more bits
// cancelled, zero included) lowers `fmin` below 2^29, and its result is
// not to be used.
//
// Band argument for a run of links: if the chain value starts at a scale in
// [-75, 56] (or is zero) and every product is zero or of scale in [-75, 56],
// each link moves the scale by at most one, so 32 links keep SL within
// [-107, 87]; callers check that once per run of 32 and take
// pzs_link_general for the run when it fails or when fmin says so.  (Runs
// of 8 / 16 / 32 measured 101 / 91 / 87 clocks per link at n = 8192: the
// check and its branch cost about as much as a few links.)
#pragma once
#include "posit_core.cuh"

namespace posit {

constexpr int PZS_ZERO_S = -(1 << 20);
constexpr int PZS_NAR_S = 1 << 20;
constexpr int PZS_BAND_LO = -75, PZS_BAND_HI = 56;  // start values and products of a run
constexpr int PZS_RUN = 32;                         // links per checked run

struct pzs {
  int s;
  int32_t m;
};

// Rounding constants of the three results of a link with larger scale SL:
// A (scale SL + 1, leading bit 30), B (SL, bit 29), C (SL - 1, rounding 2R).
// A's mask after halving is ~hA.
struct alignas(16) pzs_rtab {
  uint32_t hA, hB, hC, pA;  // 2^(p-1) - 1, and A's last kept bit
  uint32_t mB, mC, pB, pC;  // masks of the kept bits, last kept bits
};

static __device__ __forceinline__ uint32_t pzs_km(int S) { return (uint32_t)((S >> 2) ^ (S >> 31)); }

// Table entry i serves SL with SL & 255 == i; scales outside the band get
// the nearest in-band entry (never used for a result that is kept).
static __device__ __forceinline__ pzs_rtab pzs_rtab_entry(int i) {
  int SL = (int)(int8_t)(uint8_t)i;
  SL = SL < -107 ? -107 : (SL > 88 ? 88 : SL);
  pzs_rtab e;
  const uint32_t pA = 3u + pzs_km(SL + 1), pB = 2u + pzs_km(SL), pC = 2u + pzs_km(SL - 1);
  e.pA = pA; e.pB = pB; e.pC = pC;
  e.hA = (1u << (pA - 1u)) - 1u;
  e.hB = (1u << (pB - 1u)) - 1u;
  e.hC = (1u << (pC - 1u)) - 1u;
  e.mB = ~(2u * e.hB + 1u);
  e.mC = ~(2u * e.hC + 1u);
  return e;
}

static __device__ __forceinline__ pzs pzs_of(pz v) {
  if (pz_is_nar(v)) return pzs{PZS_NAR_S, 0};
  if (pz_is_zero(v)) return pzs{PZS_ZERO_S, 0};
  const uint32_t mag = (v.m & 0x7FFFFFFFu) >> 1;  // 28 significant bits: none lost
  return pzs{v.s, (int32_t)((v.m >> 31) ? 0u - mag : mag)};
}

static __device__ __forceinline__ pz pz_of(pzs v) {
  if (v.m == 0) return v.s == PZS_NAR_S ? pz_nar() : pz_zero();
  const uint32_t sign = v.m < 0 ? 0x80000000u : 0u;
  const uint32_t mag = v.m < 0 ? 0u - (uint32_t)v.m : (uint32_t)v.m;
  if (mag == (1u << 30)) return pz{v.s + 1, sign | (1u << 30)};
  return pz{v.s, sign | (mag << 1)};
}

static __device__ __forceinline__ bool pzs_in_band(pzs v) {
  return v.m == 0 ? v.s == PZS_ZERO_S : (unsigned)(v.s - PZS_BAND_LO) <= (unsigned)(PZS_BAND_HI - PZS_BAND_LO);
}

// c (+) t for every pair (NaR and zero included), through the general addition.
static __device__ __noinline__ pzs pzs_link_general(pzs c, pzs t) {
  return pzs_of(pz_add(pz_of(c), pz_of(t)));
}

static __device__ __forceinline__ void pzs_link(pzs &c, pzs t, const pzs_rtab *tab, uint32_t &fmin) {
  const int dd = c.s - t.s;
  const int SL = max(c.s, t.s);
  const uint32_t dC = (uint32_t)max(-dd, 0), dT = (uint32_t)max(dd, 0);
  int32_t aC, aT;  // arithmetic shifts; counts of 32 or more give 0 or -1
  asm("shr.s32 %0, %1, %2;" : "=r"(aC) : "r"(c.m), "r"(dC));
  asm("shr.s32 %0, %1, %2;" : "=r"(aT) : "r"(t.m), "r"(dT));
  const uint32_t R = (uint32_t)aC + (uint32_t)aT;
  // the bits shifted out (all of them from 32 on): only whether any is set
  const uint32_t st = min(__funnelshift_rc(0u, (uint32_t)c.m, dC) | __funnelshift_rc(0u, (uint32_t)t.m, dT), 1u);
  const uint4 *ep = reinterpret_cast<const uint4 *>(tab + (SL & 255));
  const uint4 e0 = ep[0], e1 = ep[1];  // hA hB hC pA, mB mC pB pC
  const uint32_t rB = R + e0.y + (((R >> e1.z) & 1u) | st);
  const uint32_t mB = rB & e1.x;
  const uint32_t sg = (uint32_t)((int32_t)R >> 31);
  const uint32_t rA = R + e0.x + (((R >> e0.w) & 1u) | st);
  const uint32_t mA = __funnelshift_r(rA, sg, 1u) & ~e0.x;  // halved with R's sign
  const uint32_t x2 = R << 1;
  const uint32_t rC = x2 + e0.z + (((x2 >> e1.w) & 1u) | st);
  const uint32_t mC = rC & e1.y;
  const bool c0 = (R + 0x40000000u) >= 0x80000000u;  // |R| >= 2^30 (R = -2^30: B, the same value)
  const bool c1 = (R + 0x20000000u) >= 0x40000000u;  // |R| >= 2^29
  c.m = (int32_t)(c0 ? mA : (c1 ? mB : mC));
  c.s = c0 ? SL + 1 : (c1 ? SL : SL - 1);
  fmin = min(fmin, R + 0x10000000u);  // below 2^29: |R| < 2^28
}

// One checked run: the links c (+) pt[0], ..., c (+) pt[cnt - 1] (N > 0: cnt =
// N, unrolled; N = 0: cnt <= PZS_RUN, rolled).  products_ok: every product is
// zero or of scale in the band (the caller's check).  The signed form runs
// when that and the start value allow it; the general addition takes the run
// (again, from its start) when they do not or when a sum cancelled two or
// more bits.
template <int N>
static __device__ __forceinline__ void pzs_run(pzs &c, const pzs *pt, int cnt, const pzs_rtab *tab,
                                               bool products_ok) {
  const pzs save = c;
  bool general = !products_ok || !pzs_in_band(save);
  if (!general) {
    uint32_t fmin = 0xFFFFFFFFu;
    if (N > 0) {
#pragma unroll
      for (int u = 0; u < N; ++u) pzs_link(c, pt[u], tab, fmin);
    } else {
#pragma unroll 4
      for (int u = 0; u < cnt; ++u) pzs_link(c, pt[u], tab, fmin);
    }
    general = fmin < 0x20000000u;
  }
  if (general) {
    c = save;
    const int k = N > 0 ? N : cnt;
    for (int u = 0; u < k; ++u) c = pzs_link_general(c, pt[u]);
  }
}

}  // namespace posit
