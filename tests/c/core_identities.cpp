// Host check of the identities that the fast forms of the GPU arithmetic in
// paper_2401_14117_gb300/csrc/posit_core.cuh rest on: each fast form must give
// the same decoded result as the general one it replaces.
//   * pz_add_serial (the dot-form chains)            == pz_add_fast
//   * pz_mul_tab, pz_mul_inband (sticky in the tie)  == pz_mul_fast
//   * pz_add_inband, pz_add_inband_blend (in band)   == pz_add_fast, through the
//     rounding (the zero scale may differ: both are far below every real scale)
//   * pz_round_apply on every in-band table row       == pz_round
//   * Rgemm's in-band multiply-add chains (operand scales in [-40, 40], start
//     in [-80, 80]) == the general multiply-add chain, at every step: the
//     in-band path relies on such chains never reaching the long-regime band
// Operands are drawn from several families (any word; near cancellation;
// near equality; |x| near 1; long regimes; exact zeros).  Usage:
//   core_identities [pairs]   -> prints one line, exit status 0 when all agree.
#include <cstdio>
#include <cstdlib>
#include <random>

#include "core_host.h"
#include "../../paper_2401_14117_gb300/csrc/posit_core.cuh"

static bool same(pz a, pz b) { return a.s == b.s && a.m == b.m; }
static bool same_value(pz a, pz b) {
  return pz_to_bits(pz_canon(a, false)) == pz_to_bits(pz_canon(b, false));
}
static bool in_band_op(pz x) { return pz_is_zero(x) || (x.s >= -40 && x.s <= 40); }

int main(int argc, char **argv) {
  const long pairs = argc > 1 ? atol(argv[1]) : 4000000;
  static pz_rtab tab[256], tin[256];
  for (int i = 0; i < 256; ++i) {
    tab[i] = pz_rtab_entry(i);
    tin[i] = pz_rtab_inband_entry(i);
  }
  std::mt19937_64 g(20240125);
  long bad_serial = 0, bad_mul = 0, bad_add_ib = 0, bad_round = 0, n_ib = 0;
  for (long it = 0; it < pairs; ++it) {
    const uint64_t r = g();
    uint32_t a = (uint32_t)r, b = (uint32_t)(r >> 32);
    switch (it % 7) {
      case 1: b = (0u - a) + (uint32_t)((int)(g() % 9) - 4); break;           // near cancellation
      case 2: b = a + (uint32_t)((int)(g() % 17) - 8); break;                  // near equality
      case 3: a = (a & 0x8FFFFFFFu) | 0x30000000u;                             // |x| near 1
              b = (b & 0x8FFFFFFFu) | ((uint32_t)(2 + g() % 4) << 28); break;
      case 4: b = (b >> (g() % 31)) ^ ((g() & 1) ? 0x80000000u : 0u); break;  // long regimes
      case 5: if (g() & 1) a = 0; else b = 0; break;                          // zeros
      default: break;
    }
    if (a == PZ_NAR_BITS || b == PZ_NAR_BITS) continue;
    const pz x = pz_decode(a), y = pz_decode(b);
    const pz add_ref = pz_add_fast(x, y), mul_ref = pz_mul_fast(x, y);
    if (!same(pz_add_serial(x, y), add_ref)) ++bad_serial;
    if (!same(pz_mul_tab(tab, x, y), mul_ref)) ++bad_mul;
    if (in_band_op(x) && in_band_op(y)) {
      ++n_ib;
      const pz p = pz_mul_inband(tin, x, y);
      if (!same_value(p, mul_ref) || (!pz_is_zero(mul_ref) && !same(p, mul_ref))) ++bad_mul;
      // an accumulator-like left operand in [-80, 80] and the rounded product
      pz c = pz_decode((uint32_t)g());
      if (pz_is_nar(c) || !(pz_is_zero(c) || (c.s >= -80 && c.s <= 80))) c = pz_one();
      const pz want = pz_add_fast(c, p);
      const pz s1 = pz_add_inband(tin, c, p), s2 = pz_add_inband_blend(tin, 0xFFFFFFFFu, c, p);
      if (!same_value(s1, want) || (!pz_is_zero(want) && !same(s1, want))) ++bad_add_ib;
      if (!same_value(s2, want) || (!pz_is_zero(want) && !same(s2, want))) ++bad_add_ib;
    }
    // the table rounding against the bit-string rule, one in-band row per pair
    const int S = (int)(g() % 217) - 108;
    const uint32_t X = (0x40000000u | (uint32_t)(g() & 0x3FFFFFFFu)) & (it & 1 ? ~0u : ~7u);
    const uint32_t sg = (g() & 1) ? 0x80000000u : 0u;
    if (!same(pz_round_apply(tin[S & 255], sg, S, X), pz_round(sg, S, X))) ++bad_round;
  }
  // accumulation chains with operands at the band's extremes: products near
  // 2^+-80 and sums that grow towards the 2^88 bound or cancel
  long bad_chain = 0, chain_steps = 0;
  const int chains = (int)(pairs / 20000) + 1;
  for (int ch = 0; ch < chains; ++ch) {
    const int K = 256 << (ch % 6);  // 256 .. 8192
    const int mode = ch % 4;
    auto operand = [&](void) {
      // a posit of scale lo..hi (or zero one time in 64), rounded from a double
      // of binade lo..hi-1 (rounding up can reach 2^hi, not beyond)
      const int lo = mode == 0 ? 30 : -40, hi = mode == 1 ? -30 : 40;
      if ((g() & 63) == 0) return pz_zero();
      const int e = lo + (int)(g() % (uint64_t)(hi - lo));
      const double v = std::ldexp(1.0 + (double)(g() >> 11) * 0x1p-53, e);
      const uint32_t w = pz_from_double((g() & 1) ? -v : v);
      return pz_decode(w);
    };
    pz accF = pz_zero(), accI = pz_zero();
    if (mode == 2) accF = accI = pz{80, 0x40000000u};          // start at 2^80
    for (int k = 0; k < K; ++k) {
      pz a = operand(), b = operand();
      if (mode == 3 && (k & 1)) { b = a; a = pz_one(); a.m ^= 0x80000000u; }  // x - x patterns
      accF = pz_add_fast(accF, pz_mul_fast(b, a));
      accI = pz_add_inband_blend(tin, 0xFFFFFFFFu, accI, pz_mul_inband(tin, b, a));
      ++chain_steps;
      if (!same_value(accF, accI)) { ++bad_chain; break; }
    }
  }
  printf("pairs %ld (in band %ld): serial add %ld, multiply %ld, in-band add %ld, rounding %ld, "
         "chains %ld mismatches (%ld chain steps)\n", pairs, n_ib, bad_serial, bad_mul,
         bad_add_ib, bad_round, bad_chain, chain_steps);
  return (bad_serial || bad_mul || bad_add_ib || bad_round || bad_chain) ? 1 : 0;
}
