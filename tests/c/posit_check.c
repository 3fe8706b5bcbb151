/*
 * posit_check.c -- independent checker for the oracle's scalar Posit(n,2)
 * operations (test code; it links against the oracle and verifies it).
 *
 * Nothing here reuses the oracle's decoding or rounding.  The checker
 *   - decodes a pattern with its own count-leading-zeros routine
 *     (Sec. 2, Eq. 1: regime run length m, k = m-1 or -m, es = 2 exponent
 *     bits, the rest fraction);
 *   - verifies, instead of computing, each rounded result r: the exact value
 *     x of the operation must lie in the rounding interval of r, whose ends
 *     are the values of the (n+1)-bit posits 2|r|-1 and 2|r|+1 (the midpoints
 *     to the neighbouring n-bit posits); x equal to an end belongs to the
 *     neighbour with the even pattern; below minpos / above maxpos saturate;
 *   - compares exact values with 256-bit integer arithmetic (sums) or with
 *     exact products of small integers (products, quotients, square roots).
 *
 * Usage:
 *   posit_check exhaustive <nbits> <op> [stride offset]
 *                                              all pairs (op: add mul div sub sqrt),
 *                                              or first operands offset + i*stride only
 *   posit_check random <op> <count> <seed>     Posit(32,2) random pairs
 *   posit_check double <count> <seed>          Posit(32,2) from double
 *   posit_check unary32 <op> <stride>          sqrt / recip over 2^32 / stride words
 *   posit_check roundtrip32 <stride>           to_double -> from_double identity
 * Prints "checked=<N> bad=<M>" and the first few failures.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include "../../oracle/posit_oracle.h"

typedef unsigned __int128 u128;

/* dyadic value: (-1)^neg * sig * 2^exp ; zero if sig == 0 */
typedef struct { int neg; uint64_t sig; int exp; } dy;

static uint32_t mask_of(int n) { return n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u); }

/* Independent decoder for n <= 33 bits: the regime run length comes from a
   count-leading-zeros of the left-aligned body (or of its complement). */
static dy value_of(int n, uint64_t p)
{
    dy v = {0, 0, 0};
    uint64_t msk = (1ull << n) - 1;
    p &= msk;
    if (p == 0) return v;
    v.neg = (int)((p >> (n - 1)) & 1);
    uint64_t a = v.neg ? ((~p + 1) & msk) : p;
    uint64_t body = a << (65 - n);       /* the n-1 bits after the sign */
    int first = (int)(body >> 63);
    uint64_t pad = ~0ull >> (n - 1);     /* ones past the end of the body */
    uint64_t run = (first ? ~body : body) | pad;
    int m = __builtin_clzll(run);        /* regime run length, <= n-1 */
    int k = first ? m - 1 : -m;
    int used = m + 1;                    /* run plus terminating bit */
    int rem = (n - 1) - used;            /* bits left for exponent, fraction */
    uint64_t tail = used >= 64 ? 0 : (body << used);
    int e = 0, fs = 0;
    if (rem >= 1) {
        e = (int)(tail >> 62);           /* missing exponent bits read as 0 */
        fs = rem > 2 ? rem - 2 : 0;
    }
    uint64_t f = fs ? ((tail << 2) >> (64 - fs)) : 0;
    v.sig = (1ull << fs) | f;
    v.exp = 4 * k + e - fs;
    return v;
}

static int msb64(uint64_t x) { return 63 - __builtin_clzll(x); }

/* compare magnitudes s1*2^e1 and s2*2^e2 (both nonzero, s < 2^64) */
static int cmp_mag(uint64_t s1, int e1, uint64_t s2, int e2)
{
    int p1 = msb64(s1) + e1, p2 = msb64(s2) + e2;
    if (p1 != p2) return p1 < p2 ? -1 : 1;
    int e = e1 < e2 ? e1 : e2;
    u128 a = (u128)s1 << (e1 - e), b = (u128)s2 << (e2 - e);
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* ---- 256-bit two's-complement integers for exact sums ---- */
typedef struct { uint64_t w[4]; } i256;

static i256 i256_from(dy v, int base) /* v * 2^-base as integer (exact) */
{
    i256 r;
    memset(&r, 0, sizeof r);
    if (v.sig == 0) return r;
    int sh = v.exp - base; /* >= 0 by choice of base */
    int word = sh / 64, bit = sh % 64;
    r.w[word] = v.sig << bit;
    if (bit && word + 1 < 4) r.w[word + 1] = v.sig >> (64 - bit);
    if (v.neg) {
        for (int i = 0; i < 4; i++) r.w[i] = ~r.w[i];
        for (int i = 0; i < 4; i++) { if (++r.w[i] != 0) break; }
    }
    return r;
}

static i256 i256_add(i256 a, i256 b)
{
    i256 r;
    unsigned carry = 0;
    for (int i = 0; i < 4; i++) {
        u128 s = (u128)a.w[i] + b.w[i] + carry;
        r.w[i] = (uint64_t)s;
        carry = (unsigned)(s >> 64);
    }
    return r;
}

static i256 i256_neg(i256 a)
{
    for (int i = 0; i < 4; i++) a.w[i] = ~a.w[i];
    for (int i = 0; i < 4; i++) { if (++a.w[i] != 0) break; }
    return a;
}

static int i256_sign(i256 a)
{
    if ((int64_t)a.w[3] < 0) return -1;
    return (a.w[0] | a.w[1] | a.w[2] | a.w[3]) ? 1 : 0;
}

/* ---- the exact operation result, compared with a dyadic m ---- */
enum { OP_ADD, OP_SUB, OP_MUL, OP_DIV, OP_SQRT, OP_RECIP };

/* sign of (x - m) where x = a op b; x and m nonzero with the same sign is
   not assumed.  For div/sqrt the caller guarantees the relevant signs. */
static int cmp_result(int op, dy a, dy b, dy m, int nbits)
{
    if (op == OP_ADD || op == OP_SUB) {
        if (op == OP_SUB) b.neg ^= 1;
        int base = -4 * (nbits + 1) + 2; /* below every lsb involved; sums stay < 2^252 */
        i256 s = i256_add(i256_from(a, base), i256_from(b, base));
        s = i256_add(s, i256_neg(i256_from(m, base)));
        return i256_sign(s);
    }
    /* remaining ops: compare signs then magnitudes */
    int xneg;
    if (op == OP_MUL) xneg = a.neg ^ b.neg;
    else if (op == OP_DIV) xneg = a.neg ^ b.neg;
    else if (op == OP_RECIP) xneg = a.neg;
    else xneg = 0;
    int sx = xneg ? -1 : 1; /* x nonzero here */
    int sm = m.sig == 0 ? 0 : (m.neg ? -1 : 1);
    if (sx != sm) return sx > sm ? 1 : -1;
    int c; /* compare |x| with |m| */
    if (op == OP_MUL)
        c = cmp_mag(a.sig * b.sig, a.exp + b.exp, m.sig, m.exp);
    else if (op == OP_DIV) /* |a|/|b| vs |m|  <=>  |a| vs |m||b| */
        c = cmp_mag(a.sig, a.exp, m.sig * b.sig, m.exp + b.exp);
    else if (op == OP_RECIP) /* 1/|a| vs |m| <=> 1 vs |m||a| */
        c = cmp_mag(1, 0, m.sig * a.sig, m.exp + a.exp);
    else /* sqrt(a) vs m  <=>  a vs m^2 */
        c = cmp_mag(a.sig, a.exp, m.sig * m.sig, 2 * m.exp);
    return xneg ? -c : c;
}

/* is r the correctly rounded posit of x = a op b ?  (x nonzero, finite) */
static int rounding_ok(int n, uint32_t r, int op, dy a, dy b)
{
    uint32_t msk = mask_of(n), nar = 1u << (n - 1);
    if (r == 0 || r == nar) return 0;
    int rneg = (r >> (n - 1)) & 1;
    uint32_t p = rneg ? ((~r + 1u) & msk) : r; /* |r| pattern */
    uint32_t maxpat = nar - 1;
    /* the result must have the sign of x: compare x with 0 */
    dy zero = {0, 0, 0};
    int sx = cmp_result(op, a, b, zero, n);
    if (sx == 0 || (sx < 0) != rneg) return 0;
    /* interval ends as signed values: lo = value(2p-1), hi = value(2p+1)
       of the (n+1)-bit format, carrying the sign of r */
    if (p > 1) {
        dy lo = value_of(n + 1, 2 * p - 1);
        lo.neg = rneg;
        int c = cmp_result(op, a, b, lo, n); /* x - lo */
        if (rneg) c = -c;                    /* |x| - |lo| */
        if (c < 0 || (c == 0 && (p & 1))) return 0;
    }
    if (p < maxpat) {
        dy hi = value_of(n + 1, 2 * p + 1);
        hi.neg = rneg;
        int c = cmp_result(op, a, b, hi, n);
        if (rneg) c = -c;
        if (c > 0 || (c == 0 && (p & 1))) return 0;
    }
    return 1;
}

static uint32_t oracle_op(int n, int op, uint32_t a, uint32_t b)
{
    switch (op) {
    case OP_ADD: return or_add(n, a, b);
    case OP_SUB: return or_sub(n, a, b);
    case OP_MUL: return or_mul(n, a, b);
    case OP_DIV: return or_div(n, a, b);
    case OP_SQRT: return or_sqrt(n, a);
    default: return or_div(n, 0x40000000u >> (32 - n), a); /* 1 / a */
    }
}

/* full check of one operation instance, including specials */
static int check_one(int n, int op, uint32_t a, uint32_t b)
{
    uint32_t msk = mask_of(n), nar = 1u << (n - 1);
    a &= msk; b &= msk;
    uint32_t r = oracle_op(n, op, a, b) & msk;
    int unary = (op == OP_SQRT || op == OP_RECIP);
    if (a == nar || (!unary && b == nar)) return r == nar;
    dy va = value_of(n, a), vb = value_of(n, b);
    switch (op) {
    case OP_ADD:
    case OP_SUB: {
        if (a == 0 && b == 0) return r == 0;
        dy nb = vb;
        if (op == OP_SUB) nb.neg ^= 1;
        /* exact zero iff the two addends have equal magnitude, opposite sign */
        if (a != 0 && b != 0 && va.neg != nb.neg &&
            cmp_mag(va.sig, va.exp, nb.sig, nb.exp) == 0)
            return r == 0;
        if (a == 0) return r == ((op == OP_SUB) ? ((~b + 1u) & msk) : b);
        if (b == 0) return r == a;
        return rounding_ok(n, r, op, va, vb);
    }
    case OP_MUL:
        if (a == 0 || b == 0) return r == 0;
        return rounding_ok(n, r, op, va, vb);
    case OP_DIV:
        if (b == 0) return r == nar;
        if (a == 0) return r == 0;
        return rounding_ok(n, r, op, va, vb);
    case OP_SQRT:
        if (a == 0) return r == 0;
        if (va.neg) return r == nar;
        return rounding_ok(n, r, op, va, vb);
    default: /* reciprocal */
        if (a == 0) return r == nar;
        return rounding_ok(n, r, op, va, vb);
    }
}

static int op_of(const char *s)
{
    if (!strcmp(s, "add")) return OP_ADD;
    if (!strcmp(s, "sub")) return OP_SUB;
    if (!strcmp(s, "mul")) return OP_MUL;
    if (!strcmp(s, "div")) return OP_DIV;
    if (!strcmp(s, "sqrt")) return OP_SQRT;
    if (!strcmp(s, "recip")) return OP_RECIP;
    fprintf(stderr, "unknown op %s\n", s);
    exit(2);
}

static uint64_t splitmix64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* random Posit(32,2) words from a few families: any word; words in the
   golden zone; words with long regimes; words next to powers of two */
static uint32_t draw_word(uint64_t *s)
{
    uint64_t z = splitmix64(s);
    uint32_t w = (uint32_t)(z >> 32);
    uint32_t sign = w & 0x80000000u;
    switch ((unsigned)(z & 3)) {
    case 0: return w;                                   /* any word */
    case 1: /* |x| roughly in [2^-8, 2^8): the golden zone */
        return (w & 0x8FFFFFFFu) | ((uint32_t)(2 + ((z >> 8) & 3)) << 28);
    case 2: { /* long regimes: tiny or huge magnitudes */
        uint32_t body = (w & 0x7FFFFFFFu) >> (1 + (unsigned)((z >> 8) % 30));
        if ((z >> 16) & 1) body = 0x7FFFFFFFu - body;
        if (body == 0) body = 1;
        return sign ? (0u - body) : body;
    }
    default: /* few fraction bits set: exact results and ties */
        return (w & 0xFFFC0000u) | ((w >> 5) & 1u);
    }
}

static long report(long checked, long bad)
{
    printf("checked=%ld bad=%ld\n", checked, bad);
    return bad;
}

int main(int argc, char **argv)
{
    if (argc < 2) { fprintf(stderr, "usage\n"); return 2; }
    long checked = 0, bad = 0;
    if (!strcmp(argv[1], "exhaustive")) {
        int n = atoi(argv[2]);
        int op = op_of(argv[3]);
        uint32_t count = 1u << n;
        int unary = (op == OP_SQRT || op == OP_RECIP);
        uint32_t bcount = unary ? 1u : count;
        /* optional slice: only first operands a = offset, offset + stride, ... */
        int64_t stride = argc > 5 ? atoll(argv[4]) : 1, offset = argc > 5 ? atoll(argv[5]) : 0;
        if (stride < 1 || offset < 0 || offset >= stride) { fprintf(stderr, "slice\n"); return 2; }
        int64_t slices = ((int64_t)count - offset + stride - 1) / stride;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : checked, bad)
        for (int64_t si = 0; si < slices; si++) {
            int64_t ai = offset + si * stride;
            for (uint32_t b = 0; b < bcount; b++) {
                checked++;
                if (!check_one(n, op, (uint32_t)ai, b)) {
                    bad++;
                    if (bad < 5) {
#pragma omp critical
                        printf("FAIL n=%d op=%s a=0x%x b=0x%x r=0x%x\n", n, argv[3],
                               (unsigned)ai, b, oracle_op(n, op, (uint32_t)ai, b));
                    }
                }
            }
        }
        return report(checked, bad) != 0;
    }
    if (!strcmp(argv[1], "random")) {
        int op = op_of(argv[2]);
        long count = atol(argv[3]);
        uint64_t seed = strtoull(argv[4], 0, 10);
#pragma omp parallel for schedule(static) reduction(+ : checked, bad)
        for (long i = 0; i < count; i++) {
            uint64_t s = seed * 0x100000001B3ull + (uint64_t)i * 0x9E3779B97F4A7C15ull;
            uint32_t a = draw_word(&s), b = draw_word(&s);
            if (splitmix64(&s) & 1) b = (b & 0xF80FFFFFu) | (a & 0x07F00000u); /* near scales */
            checked++;
            if (!check_one(32, op, a, b)) {
                bad++;
                if (bad < 5) {
#pragma omp critical
                    printf("FAIL op=%s a=0x%08x b=0x%08x r=0x%08x\n", argv[2], a, b,
                           oracle_op(32, op, a, b));
                }
            }
        }
        return report(checked, bad) != 0;
    }
    if (!strcmp(argv[1], "double")) {
        long count = atol(argv[2]);
        uint64_t seed = strtoull(argv[3], 0, 10);
#pragma omp parallel for schedule(static) reduction(+ : checked, bad)
        for (long i = 0; i < count; i++) {
            uint64_t s = seed + (uint64_t)i * 0x9E3779B97F4A7C15ull;
            uint64_t z = splitmix64(&s);
            double x;
            if (i & 1) { memcpy(&x, &z, 8); } /* any finite double */
            else x = ldexp((double)(z >> 11) * 0x1p-53 * 2 - 1, (int)(splitmix64(&s) % 97) - 48);
            if (isnan(x) || isinf(x) || x == 0) continue;
            uint32_t r = or_from_double(32, x);
            /* x as a dyadic: x = a * 1 with op MUL against the word for 1 */
            int ex;
            double mm = frexp(fabs(x), &ex);
            dy a = {x < 0, (uint64_t)ldexp(mm, 53), ex - 53};
            dy one = {0, 1, 0};
            checked++;
            if (!rounding_ok(32, r, OP_MUL, a, one)) {
                bad++;
                if (bad < 5) {
#pragma omp critical
                    printf("FAIL double %.17g -> 0x%08x\n", x, r);
                }
            }
        }
        return report(checked, bad) != 0;
    }
    if (!strcmp(argv[1], "unary32")) {
        int op = op_of(argv[2]);
        uint64_t stride = strtoull(argv[3], 0, 10);
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : checked, bad)
        for (int64_t w = 0; w < (int64_t)1 << 32; w += (int64_t)stride) {
            checked++;
            if (!check_one(32, op, (uint32_t)w, 0)) {
                bad++;
                if (bad < 5) {
#pragma omp critical
                    printf("FAIL %s 0x%08x -> 0x%08x\n", argv[2], (unsigned)w,
                           oracle_op(32, op, (uint32_t)w, 0));
                }
            }
        }
        return report(checked, bad) != 0;
    }
    if (!strcmp(argv[1], "roundtrip32")) {
        uint64_t stride = strtoull(argv[2], 0, 10);
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : checked, bad)
        for (int64_t w = 0; w < (int64_t)1 << 32; w += (int64_t)stride) {
            uint32_t p = (uint32_t)w;
            if (p == 0x80000000u) continue;
            double d = or_to_double(32, p);
            dy v = value_of(32, p);
            double want = ldexp((double)v.sig, v.exp) * (v.neg ? -1.0 : 1.0);
            checked++;
            if (d != want || or_from_double(32, d) != p) {
                bad++;
                if (bad < 5) {
#pragma omp critical
                    printf("FAIL roundtrip 0x%08x\n", p);
                }
            }
        }
        return report(checked, bad) != 0;
    }
    fprintf(stderr, "unknown mode\n");
    return 2;
}
