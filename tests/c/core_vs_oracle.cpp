// The GPU arithmetic's general operations, compiled on the host, against the
// oracle's (linked from its C library): decode -> one rounded operation ->
// encode must give the oracle's word for add, sub, mul, div and sqrt, and the
// FP64 conversion must agree too.  Operands come from several families (any
// word, |x| near 1, long regimes, few fraction bits, cancellation, the special
// words).  Usage: core_vs_oracle [cases]  -> one line, exit status 0 when all
// agree.
#include <cstdio>
#include <cstdlib>
#include <random>

#include "core_host.h"
#include "../../paper_2401_14117_gb300/csrc/posit_core.cuh"

extern "C" {
uint32_t or_add(int n, uint32_t a, uint32_t b);
uint32_t or_sub(int n, uint32_t a, uint32_t b);
uint32_t or_mul(int n, uint32_t a, uint32_t b);
uint32_t or_div(int n, uint32_t a, uint32_t b);
uint32_t or_sqrt(int n, uint32_t a);
uint32_t or_from_double(int n, double x);
}

static uint32_t word(std::mt19937_64 &g, int fam) {
  uint32_t w = (uint32_t)g();
  switch (fam) {
    case 1: return (w & 0x8FFFFFFFu) | 0x30000000u;                          // |x| near 1
    case 2: return (w >> (g() % 31)) ^ ((g() & 1) ? 0x80000000u : 0u) ^ 0u;  // long regimes
    case 3: return w & 0xFFFFF000u;                                            // few fraction bits
    case 4: { const uint32_t s[] = {0u, 0x80000000u, 1u, 0x7FFFFFFFu, 0x40000000u, 0xC0000000u,
                                    0xFFFFFFFFu, 0x80000001u};
              return s[g() % 8]; }                                             // special words
    default: return w;
  }
}

int main(int argc, char **argv) {
  const long cases = argc > 1 ? atol(argv[1]) : 1000000;
  std::mt19937_64 g(20240128);
  long bad[6] = {0, 0, 0, 0, 0, 0};
  for (long it = 0; it < cases; ++it) {
    uint32_t a = word(g, (int)(it % 5)), b = word(g, (int)((it / 5) % 5));
    if (it % 11 == 7) b = (0u - a) + (uint32_t)((int)(g() % 9) - 4);  // cancellation
    const pz x = pz_decode(a), y = pz_decode(b);
    if (pz_to_bits(pz_add(x, y)) != or_add(32, a, b)) ++bad[0];
    if (pz_to_bits(pz_sub(x, y)) != or_sub(32, a, b)) ++bad[1];
    if (pz_to_bits(pz_mul(x, y)) != or_mul(32, a, b)) ++bad[2];
    if (pz_to_bits(pz_div(x, y)) != or_div(32, a, b)) ++bad[3];
    if (pz_to_bits(pz_sqrt(x)) != or_sqrt(32, a)) ++bad[4];
    // FP64 -> posit: random doubles over a wide exponent range
    const double v = std::ldexp((double)(g() >> 11) * 0x1p-53 * ((g() & 1) ? 1.0 : -1.0),
                                (int)(g() % 400) - 200);
    if (pz_from_double(v) != or_from_double(32, v)) ++bad[5];
  }
  printf("cases %ld mismatches: add %ld sub %ld mul %ld div %ld sqrt %ld from_double %ld\n", cases,
         bad[0], bad[1], bad[2], bad[3], bad[4], bad[5]);
  long tot = 0;
  for (long v : bad) tot += v;
  return tot ? 1 : 0;
}
