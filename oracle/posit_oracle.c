/*
 * posit_oracle.c -- plain, slow CPU oracle for Posit(n,2) arithmetic and the
 * Posit(32,2) routines Rgemm, Rgetrf, Rpotrf, Rgetrs and Rpotrs.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load it; the CUDA library shares
 * no code with it and never calls it.
 *
 * Every scalar operation is "compute the exact result, then round it once":
 *   - decode    : Sec. 2, Eq. 1.  x = (-1)^s * u^k * 2^e * 1.f with
 *                 u = 2^(2^es) = 16; k from the regime run length (Sec. 2,
 *                 the k(r) paragraph); f_s = n - m - es - 2 fraction bits.
 *   - mul, div, sqrt, add: exact (div and sqrt carry a sticky flag meaning
 *                 "the true value lies strictly between sig and sig+1 units"),
 *                 Sec. 2 pre-/post-processing paragraph: decode, operate in an
 *                 internal format, re-encode the regime and round with the new
 *                 f_s.
 *   - rounding  : the paper does not state it.  Reading used here: build the
 *                 exact value's infinite posit bit string (regime | exponent |
 *                 fraction), keep the n-1 bits after the sign and round to
 *                 nearest, ties to the even pattern; never round a nonzero to
 *                 0 or to NaR (values beyond maxpos give maxpos, below minpos
 *                 give minpos).  Zero is 0x0, NaR is 0x80..0; any operation
 *                 with NaR, x/0 and sqrt(x<0) give NaR.
 *
 * The LAPACK routines follow the reference-BLAS/LAPACK loop orders the paper
 * reuses through MPLAPACK (Sec. 3), with one rounding after every multiply
 * and every add (no fused operations):
 *   Rgemm   c <- beta (x) c (c <- 0 if beta = 0); then for l ascending:
 *           t <- alpha (x) op(B)_lj ; c <- c (+) (t (x) op(A)_il).
 *   Rgetrf  per column: pivot = first row of largest |a| (two's-complement
 *           absolute value compared as unsigned, so NaR is largest), swap,
 *           scale by r = 1 (/) pivot, rank-1 update a_ik <- a_ik (-) l_i u_k.
 *   Rpotrf  per column: sqrt of the diagonal, scale by its reciprocal,
 *           update of the remaining lower (or upper) triangle.
 *   Rgetrs / Rpotrs: row swaps, then the reference-trsm substitution orders.
 */
#include "posit_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* exact values                                                               */
/* ------------------------------------------------------------------------ */

enum { XZERO = 0, XFIN = 1, XNAR = 2 };

/* value = (-1)^neg * sig * 2^exp; if sticky, the true magnitude lies
   strictly between sig*2^exp and (sig+1)*2^exp. */
typedef struct {
    int cls;
    int neg;
    int sticky;
    int64_t exp;
    u128 sig;
} xval;

static uint32_t word_mask(int n) { return n >= 32 ? 0xFFFFFFFFu : ((1u << n) - 1u); }
static uint32_t nar_word(int n) { return 1u << (n - 1); }

static int msb128(u128 x) /* position of the leading one, x != 0 */
{
    uint64_t hi = (uint64_t)(x >> 64), lo = (uint64_t)x;
    if (hi) return 127 - __builtin_clzll(hi);
    return 63 - __builtin_clzll(lo);
}

static int64_t floor_div4(int64_t s) { return s >= 0 ? s / 4 : -((-s + 3) / 4); }

/* Decode an n-bit posit (Sec. 2, Eq. 1).  The sign is removed first by a
   two's-complement negation; the regime is then the run of bits equal to the
   first bit after the sign: m ones give k = m-1, m zeros give k = -m.  The
   terminating bit is skipped, then es = 2 exponent bits (missing bits are
   zero), then the remaining f_s bits are the fraction. */
static xval decode(int n, uint32_t p)
{
    xval v;
    memset(&v, 0, sizeof v);
    p &= word_mask(n);
    if (p == 0) { v.cls = XZERO; return v; }
    if (p == nar_word(n)) { v.cls = XNAR; return v; }
    v.cls = XFIN;
    v.neg = (int)((p >> (n - 1)) & 1u);
    if (v.neg) p = (0u - p) & word_mask(n);
    int i = n - 2;
    int first = (int)((p >> i) & 1u);
    int m = 0;
    while (i >= 0 && (int)((p >> i) & 1u) == first) { m++; i--; }
    int k = first ? m - 1 : -m;
    i--; /* terminating bit of the regime (may lie past the end) */
    int e = 0;
    for (int j = 0; j < 2; j++) {
        e <<= 1;
        if (i >= 0) { e |= (int)((p >> i) & 1u); i--; }
    }
    int fs = i + 1 > 0 ? i + 1 : 0;
    uint32_t f = fs ? (p & ((1u << fs) - 1u)) : 0u;
    v.sig = ((u128)1 << fs) | f;
    v.exp = 4 * (int64_t)k + e - fs;
    return v;
}

/* Round an exact value to n bits by the bit-string rule described at the top
   of this file. */
static uint32_t encode(int n, xval v)
{
    if (v.cls == XZERO) return 0;
    if (v.cls == XNAR) return nar_word(n);
    int b = msb128(v.sig);
    int64_t S = v.exp + b; /* 2^S <= |x| < 2^(S+1) */
    int64_t k = floor_div4(S);
    int e = (int)(S - 4 * k);
    int sticky = v.sticky;
    /* A regime longer than the word just repeats its bit; clamping |k| to
       n+2 keeps the same first n+1 bits (all-equal run) and the same
       rounding, while keeping the string inside 128 bits. */
    if (k > n + 2) { k = n + 2; sticky = 1; }
    if (k < -(n + 2)) { k = -(n + 2); sticky = 1; }
    /* fraction: the b bits of sig below its leading one; bits past 64 only
       matter as sticky (at most 31 bits are kept plus one guard bit) */
    u128 frac = v.sig - ((u128)1 << b);
    int fb = b;
    if (fb > 64) {
        int drop = fb - 64;
        if (frac & (((u128)1 << drop) - 1)) sticky = 1;
        frac >>= drop;
        fb = 64;
    }
    u128 reg;
    int L; /* regime length including its terminating bit */
    if (k >= 0) { L = (int)k + 2; reg = (((u128)1 << (k + 1)) - 1) << 1; }
    else        { L = 1 - (int)k; reg = 1; }
    int T = L + 2 + fb; /* <= 38 + 2 + 64 bits */
    u128 str = (reg << (2 + fb)) | ((u128)e << fb) | frac;
    int keep = n - 1;
    uint64_t p;
    int guard;
    if (T >= keep + 1) {
        int rest = T - keep - 1; /* bits after the guard bit */
        p = (uint64_t)(str >> (rest + 1));
        guard = (int)((str >> rest) & 1);
        if (rest > 0 && (str & (((u128)1 << rest) - 1))) sticky = 1;
    } else {
        p = (uint64_t)(str << (keep - T)); /* short string: pad with zeros */
        guard = 0;
    }
    if (guard && (sticky || (p & 1u))) p += 1;
    uint64_t maxpos = ((uint64_t)1 << keep) - 1;
    if (p > maxpos) p = maxpos; /* never round up into NaR */
    if (p == 0) p = 1;          /* never round a nonzero value to zero */
    uint32_t w = (uint32_t)p;
    return v.neg ? ((0u - w) & word_mask(n)) : w;
}

static xval x_zero(void) { xval v; memset(&v, 0, sizeof v); v.cls = XZERO; return v; }
static xval x_nar(void)  { xval v; memset(&v, 0, sizeof v); v.cls = XNAR;  return v; }

static xval x_mul(xval a, xval b)
{
    if (a.cls == XNAR || b.cls == XNAR) return x_nar();
    if (a.cls == XZERO || b.cls == XZERO) return x_zero();
    xval r;
    memset(&r, 0, sizeof r);
    r.cls = XFIN;
    r.neg = a.neg ^ b.neg;
    r.sig = a.sig * b.sig; /* < 2^56: exact */
    r.exp = a.exp + b.exp;
    return r;
}

static xval x_add(xval a, xval b)
{
    if (a.cls == XNAR || b.cls == XNAR) return x_nar();
    if (a.cls == XZERO) return b;
    if (b.cls == XZERO) return a;
    if (a.exp < b.exp) { xval t = a; a = b; b = t; }
    int64_t d = a.exp - b.exp;
    xval r;
    memset(&r, 0, sizeof r);
    r.cls = XFIN;
    if (d <= 99) {
        /* both significands are below 2^28, so a.sig << d < 2^127: exact */
        u128 A = a.sig << d, B = b.sig;
        r.exp = b.exp;
        if (a.neg == b.neg)  { r.sig = A + B; r.neg = a.neg; }
        else if (A > B)      { r.sig = A - B; r.neg = a.neg; }
        else if (B > A)      { r.sig = B - A; r.neg = b.neg; }
        else return x_zero();
    } else {
        /* |b| < 2^(b.exp+28) < 2^(a.exp-71): less than one unit of
           2^(a.exp-71), so it only decides the sticky side */
        u128 A = a.sig << 71;
        r.exp = a.exp - 71;
        r.neg = a.neg;
        r.sticky = 1;
        r.sig = (a.neg == b.neg) ? A : A - 1;
    }
    return r;
}

static xval x_div(xval a, xval b)
{
    if (a.cls == XNAR || b.cls == XNAR || b.cls == XZERO) return x_nar();
    if (a.cls == XZERO) return x_zero();
    xval r;
    memset(&r, 0, sizeof r);
    r.cls = XFIN;
    r.neg = a.neg ^ b.neg;
    u128 N = a.sig << 96; /* < 2^124 */
    r.sig = N / b.sig;    /* >= 2^68 */
    r.sticky = (N % b.sig) != 0;
    r.exp = a.exp - b.exp - 96;
    return r;
}

static u128 isqrt128(u128 N) /* floor(sqrt(N)), N < 2^126 */
{
    u128 r = 0;
    for (int bit = 63; bit >= 0; bit--) {
        u128 t = r | ((u128)1 << bit);
        if (t * t <= N) r = t;
    }
    return r;
}

static xval x_sqrt(xval a)
{
    if (a.cls == XNAR) return x_nar();
    if (a.cls == XZERO) return x_zero();
    if (a.neg) return x_nar();
    u128 N = a.sig;
    int64_t ex = a.exp;
    if (ex & 1) { N <<= 1; ex -= 1; }
    N <<= 96; /* < 2^125 */
    ex -= 96;
    xval r;
    memset(&r, 0, sizeof r);
    r.cls = XFIN;
    r.sig = isqrt128(N); /* >= 2^48 */
    r.sticky = r.sig * r.sig != N;
    r.exp = ex / 2;
    return r;
}

/* ------------------------------------------------------------------------ */
/* scalar API                                                                 */
/* ------------------------------------------------------------------------ */

uint32_t or_add(int n, uint32_t a, uint32_t b) { return encode(n, x_add(decode(n, a), decode(n, b))); }
uint32_t or_mul(int n, uint32_t a, uint32_t b) { return encode(n, x_mul(decode(n, a), decode(n, b))); }
uint32_t or_div(int n, uint32_t a, uint32_t b) { return encode(n, x_div(decode(n, a), decode(n, b))); }
uint32_t or_sqrt(int n, uint32_t a)            { return encode(n, x_sqrt(decode(n, a))); }

uint32_t or_neg(int n, uint32_t a) { return (0u - a) & word_mask(n); }

uint32_t or_sub(int n, uint32_t a, uint32_t b)
{
    xval nb = decode(n, b);
    if (nb.cls == XFIN) nb.neg ^= 1;
    return encode(n, x_add(decode(n, a), nb));
}

uint32_t or_from_double(int n, double x)
{
    if (isnan(x) || isinf(x)) return nar_word(n);
    if (x == 0.0) return 0;
    int ex;
    double m = frexp(fabs(x), &ex); /* |x| = m * 2^ex, 0.5 <= m < 1 */
    xval v;
    memset(&v, 0, sizeof v);
    v.cls = XFIN;
    v.neg = x < 0;
    v.sig = (u128)(uint64_t)ldexp(m, 53); /* exact 53-bit integer */
    v.exp = (int64_t)ex - 53;
    return encode(n, v);
}

double or_to_double(int n, uint32_t p)
{
    xval v = decode(n, p);
    if (v.cls == XZERO) return 0.0;
    if (v.cls == XNAR) return NAN;
    double r = ldexp((double)(uint64_t)v.sig, (int)v.exp); /* exact */
    return v.neg ? -r : r;
}

int or_decode(int n, uint32_t p, int *neg, int *scale, uint32_t *frac, int *fbits)
{
    xval v = decode(n, p);
    *neg = 0; *scale = 0; *frac = 0; *fbits = 0;
    if (v.cls != XFIN) return v.cls;
    int b = msb128(v.sig);
    *neg = v.neg;
    *scale = (int)(v.exp + b);
    *fbits = b;
    *frac = (uint32_t)(v.sig - ((u128)1 << b));
    return XFIN;
}

void or_elementwise(int n, int op, const uint32_t *a, const uint32_t *b,
                    uint32_t *out, int64_t count)
{
#pragma omp parallel for schedule(static) if (count > 20000)
    for (int64_t i = 0; i < count; i++) {
        switch (op) {
        case 0: out[i] = or_add(n, a[i], b[i]); break;
        case 1: out[i] = or_sub(n, a[i], b[i]); break;
        case 2: out[i] = or_mul(n, a[i], b[i]); break;
        case 3: out[i] = or_div(n, a[i], b[i]); break;
        default: out[i] = or_sqrt(n, a[i]); break;
        }
    }
}

void or_from_double_array(int n, const double *x, uint32_t *out, int64_t count)
{
#pragma omp parallel for schedule(static) if (count > 20000)
    for (int64_t i = 0; i < count; i++) out[i] = or_from_double(n, x[i]);
}

void or_to_double_array(int n, const uint32_t *p, double *out, int64_t count)
{
#pragma omp parallel for schedule(static) if (count > 20000)
    for (int64_t i = 0; i < count; i++) out[i] = or_to_double(n, p[i]);
}

/* ------------------------------------------------------------------------ */
/* Posit(32,2) BLAS / LAPACK                                                  */
/* ------------------------------------------------------------------------ */

#define P32 32
#define ONE32 0x40000000u

static uint32_t padd(uint32_t a, uint32_t b) { return or_add(P32, a, b); }
static uint32_t psub(uint32_t a, uint32_t b) { return or_sub(P32, a, b); }
static uint32_t pmul(uint32_t a, uint32_t b) { return or_mul(P32, a, b); }
static uint32_t pdiv(uint32_t a, uint32_t b) { return or_div(P32, a, b); }

/* |a| as the two's-complement absolute value of the word, compared as an
   unsigned integer (posit order equals integer order; NaR = 0x80000000 is
   the largest). */
static uint32_t absword(uint32_t a) { return (a >> 31) ? (0u - a) : a; }

void or_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define AT(M, ld, i, j) (M)[(int64_t)(i) + (int64_t)(j) * (ld)]

/* Eq. GEMM_DEF: C = alpha op(A) op(B) + beta C, in the reference-BLAS order
   described at the top of this file, applied to every op(A)/op(B) pair.
   alpha = 0 or k = 0 leaves C = beta C without reading A or B. */
void or_rgemm(char transa, char transb, int64_t m, int64_t n, int64_t k,
              uint32_t alpha, const uint32_t *A, int64_t lda,
              const uint32_t *B, int64_t ldb, uint32_t beta,
              uint32_t *C, int64_t ldc)
{
    int ta = (transa == 'T' || transa == 't' || transa == 'C' || transa == 'c');
    int tb = (transb == 'T' || transb == 't' || transb == 'C' || transb == 'c');
#pragma omp parallel for schedule(dynamic, 1) if (n > 1 && m * n * (k + 1) > 100000)
    for (int64_t j = 0; j < n; j++) {
        for (int64_t i = 0; i < m; i++) {
            uint32_t c = AT(C, ldc, i, j);
            if (beta == 0) c = 0;
            else if (beta != ONE32) c = pmul(beta, c);
            if (alpha != 0) {
                for (int64_t l = 0; l < k; l++) {
                    uint32_t b = tb ? AT(B, ldb, j, l) : AT(B, ldb, l, j);
                    uint32_t a = ta ? AT(A, lda, l, i) : AT(A, lda, i, l);
                    uint32_t t = pmul(alpha, b);
                    c = padd(c, pmul(t, a));
                }
            }
            AT(C, ldc, i, j) = c;
        }
    }
}

static void swap_rows(uint32_t *A, int64_t lda, int64_t r1, int64_t r2,
                      int64_t c0, int64_t c1)
{
    if (r1 == r2) return;
    for (int64_t c = c0; c < c1; c++) {
        uint32_t t = AT(A, lda, r1, c);
        AT(A, lda, r1, c) = AT(A, lda, r2, c);
        AT(A, lda, r2, c) = t;
    }
}

/* one column step of LU restricted to columns [c0, c1): pivot search in
   column col, swap inside [c0, c1), scaling, rank-1 update of columns
   (col, c1).  Returns 1 if the pivot was zero. */
static int lu_column_step(int64_t m, uint32_t *A, int64_t lda, int32_t *ipiv,
                          int64_t col, int64_t c0, int64_t c1)
{
    int64_t p = col;
    uint32_t best = absword(AT(A, lda, col, col));
    for (int64_t i = col + 1; i < m; i++) {
        uint32_t w = absword(AT(A, lda, i, col));
        if (w > best) { best = w; p = i; }
    }
    ipiv[col] = (int32_t)(p + 1);
    int zero = AT(A, lda, p, col) == 0;
    if (!zero) {
        swap_rows(A, lda, col, p, c0, c1);
        uint32_t r = pdiv(ONE32, AT(A, lda, col, col));
        for (int64_t i = col + 1; i < m; i++)
            AT(A, lda, i, col) = pmul(AT(A, lda, i, col), r);
    }
#pragma omp parallel for schedule(static) if ((c1 - col) * (m - col) > 50000)
    for (int64_t kk = col + 1; kk < c1; kk++) {
        uint32_t u = AT(A, lda, col, kk);
        for (int64_t i = col + 1; i < m; i++)
            AT(A, lda, i, kk) = psub(AT(A, lda, i, kk), pmul(AT(A, lda, i, col), u));
    }
    return zero;
}

int or_rgetrf(int64_t m, int64_t n, uint32_t *A, int64_t lda, int32_t *ipiv)
{
    int info = 0;
    int64_t mn = m < n ? m : n;
    for (int64_t col = 0; col < mn; col++) {
        int zero = lu_column_step(m, A, lda, ipiv, col, 0, n);
        if (zero && info == 0) info = (int)(col + 1);
    }
    return info;
}

int or_rgetrf_blocked(int64_t m, int64_t n, uint32_t *A, int64_t lda,
                      int32_t *ipiv, int64_t nb)
{
    int info = 0;
    int64_t mn = m < n ? m : n;
    if (nb < 1) nb = 1;
    for (int64_t j = 0; j < mn; j += nb) {
        int64_t jb = (mn - j) < nb ? (mn - j) : nb;
        /* panel: columns [j, j+jb) */
        for (int64_t col = j; col < j + jb; col++) {
            int zero = lu_column_step(m, A, lda, ipiv, col, j, j + jb);
            if (zero && info == 0) info = (int)(col + 1);
        }
        /* the panel's row swaps on the columns left and right of it */
        for (int64_t col = j; col < j + jb; col++) {
            int64_t p = ipiv[col] - 1;
            swap_rows(A, lda, col, p, 0, j);
            swap_rows(A, lda, col, p, j + jb, n);
        }
        if (j + jb < n) {
            /* U12 <- L11^-1 A12 (unit lower, forward substitution) */
#pragma omp parallel for schedule(static) if ((n - j - jb) * jb * jb > 50000)
            for (int64_t kk = j + jb; kk < n; kk++)
                for (int64_t c = j + 1; c < j + jb; c++)
                    for (int64_t col = j; col < c; col++)
                        AT(A, lda, c, kk) = psub(AT(A, lda, c, kk),
                                                 pmul(AT(A, lda, c, col), AT(A, lda, col, kk)));
            /* A22 <- A22 - L21 U12 through Rgemm, alpha = -1, beta = 1 */
            if (j + jb < m)
                or_rgemm('N', 'N', m - j - jb, n - j - jb, jb, 0xC0000000u,
                         &AT(A, lda, j + jb, j), lda, &AT(A, lda, j, j + jb), lda,
                         ONE32, &AT(A, lda, j + jb, j + jb), lda);
        }
    }
    return info;
}

/* A = P L U (LAPACK convention).  trans 'N': solve A X = B; 'T': A^T X = B. */
void or_rgetrs(char trans, int64_t n, int64_t nrhs, const uint32_t *A,
               int64_t lda, const int32_t *ipiv, uint32_t *B, int64_t ldb)
{
    int tr = (trans == 'T' || trans == 't' || trans == 'C' || trans == 'c');
#pragma omp parallel for schedule(dynamic, 1) if (nrhs > 1 && n * n * nrhs > 100000)
    for (int64_t r = 0; r < nrhs; r++) {
        uint32_t *b = B + r * ldb;
        if (!tr) {
            for (int64_t i = 0; i < n; i++) {
                int64_t p = ipiv[i] - 1;
                uint32_t t = b[i]; b[i] = b[p]; b[p] = t;
            }
            /* L y = b, unit lower: element i gets j = 0..i-1 ascending */
            for (int64_t i = 0; i < n; i++)
                for (int64_t j = 0; j < i; j++)
                    b[i] = psub(b[i], pmul(AT(A, lda, i, j), b[j]));
            /* U x = y: element i gets k = n-1..i+1 descending, then / u_ii */
            for (int64_t i = n - 1; i >= 0; i--) {
                for (int64_t k = n - 1; k > i; k--)
                    b[i] = psub(b[i], pmul(AT(A, lda, i, k), b[k]));
                b[i] = pdiv(b[i], AT(A, lda, i, i));
            }
        } else {
            /* U^T y = b: ascending dot form, then / u_ii */
            for (int64_t i = 0; i < n; i++) {
                for (int64_t k = 0; k < i; k++)
                    b[i] = psub(b[i], pmul(AT(A, lda, k, i), b[k]));
                b[i] = pdiv(b[i], AT(A, lda, i, i));
            }
            /* L^T z = y, unit: i descending, k = i+1..n-1 ascending */
            for (int64_t i = n - 1; i >= 0; i--)
                for (int64_t k = i + 1; k < n; k++)
                    b[i] = psub(b[i], pmul(AT(A, lda, k, i), b[k]));
            /* x = P z: the swaps in reverse order */
            for (int64_t i = n - 1; i >= 0; i--) {
                int64_t p = ipiv[i] - 1;
                uint32_t t = b[i]; b[i] = b[p]; b[p] = t;
            }
        }
    }
}

/* Cholesky column step j restricted to rows/columns below `lim` (for the
   blocked form); returns 1 if the diagonal was not positive. */
static int chol_lower_step(int64_t n, uint32_t *A, int64_t lda, int64_t j, int64_t lim)
{
    uint32_t d = AT(A, lda, j, j);
    if ((int32_t)d <= 0) return 1; /* d <= 0 or NaR */
    uint32_t s = or_sqrt(P32, d);
    AT(A, lda, j, j) = s;
    uint32_t r = pdiv(ONE32, s);
    for (int64_t i = j + 1; i < n; i++) AT(A, lda, i, j) = pmul(AT(A, lda, i, j), r);
#pragma omp parallel for schedule(dynamic, 8) if ((lim - j) * (n - j) > 50000)
    for (int64_t k = j + 1; k < lim; k++) {
        uint32_t akj = AT(A, lda, k, j);
        for (int64_t i = k; i < n; i++)
            AT(A, lda, i, k) = psub(AT(A, lda, i, k), pmul(AT(A, lda, i, j), akj));
    }
    return 0;
}

static int chol_upper_step(int64_t n, uint32_t *A, int64_t lda, int64_t j, int64_t lim)
{
    uint32_t d = AT(A, lda, j, j);
    if ((int32_t)d <= 0) return 1;
    uint32_t s = or_sqrt(P32, d);
    AT(A, lda, j, j) = s;
    uint32_t r = pdiv(ONE32, s);
    for (int64_t k = j + 1; k < n; k++) AT(A, lda, j, k) = pmul(AT(A, lda, j, k), r);
#pragma omp parallel for schedule(dynamic, 8) if ((lim - j) * (n - j) > 50000)
    for (int64_t k = j + 1; k < n; k++) {
        uint32_t ajk = AT(A, lda, j, k);
        int64_t iend = k < lim - 1 ? k : lim - 1;
        for (int64_t i = j + 1; i <= iend; i++)
            AT(A, lda, i, k) = psub(AT(A, lda, i, k), pmul(AT(A, lda, j, i), ajk));
    }
    return 0;
}

int or_rpotrf(char uplo, int64_t n, uint32_t *A, int64_t lda)
{
    int up = (uplo == 'U' || uplo == 'u');
    for (int64_t j = 0; j < n; j++) {
        int bad = up ? chol_upper_step(n, A, lda, j, n) : chol_lower_step(n, A, lda, j, n);
        if (bad) return (int)(j + 1);
    }
    return 0;
}

/* Blocked right-looking Cholesky: factor the nb x nb diagonal block and the
   panel below (or right of) it column by column, then update the trailing
   triangle through Rgemm (alpha = -1, beta = 1), keeping only the lower
   (upper) triangle of each trailing column. */
int or_rpotrf_blocked(char uplo, int64_t n, uint32_t *A, int64_t lda, int64_t nb)
{
    int up = (uplo == 'U' || uplo == 'u');
    if (nb < 1) nb = 1;
    for (int64_t j = 0; j < n; j += nb) {
        int64_t jb = (n - j) < nb ? (n - j) : nb;
        for (int64_t c = j; c < j + jb; c++) {
            int bad = up ? chol_upper_step(n, A, lda, c, j + jb)
                         : chol_lower_step(n, A, lda, c, j + jb);
            if (bad) return (int)(c + 1);
        }
        int64_t t0 = j + jb;
        if (t0 >= n) continue;
        /* trailing triangle, one column (row) at a time through Rgemm */
        for (int64_t k = t0; k < n; k++) {
            if (!up)
                or_rgemm('N', 'T', n - k, 1, jb, 0xC0000000u,
                         &AT(A, lda, k, j), lda, &AT(A, lda, k, j), lda,
                         ONE32, &AT(A, lda, k, k), lda);
            else
                or_rgemm('T', 'N', 1, n - k, jb, 0xC0000000u,
                         &AT(A, lda, j, k), lda, &AT(A, lda, j, k), lda,
                         ONE32, &AT(A, lda, k, k), lda);
        }
    }
    return 0;
}

void or_rpotrs(char uplo, int64_t n, int64_t nrhs, const uint32_t *A,
               int64_t lda, uint32_t *B, int64_t ldb)
{
    int up = (uplo == 'U' || uplo == 'u');
#pragma omp parallel for schedule(dynamic, 1) if (nrhs > 1 && n * n * nrhs > 100000)
    for (int64_t r = 0; r < nrhs; r++) {
        uint32_t *b = B + r * ldb;
        if (!up) {
            /* L y = b: j ascending, then / l_ii */
            for (int64_t i = 0; i < n; i++) {
                for (int64_t j = 0; j < i; j++)
                    b[i] = psub(b[i], pmul(AT(A, lda, i, j), b[j]));
                b[i] = pdiv(b[i], AT(A, lda, i, i));
            }
            /* L^T x = y: i descending, k = i+1..n-1 ascending, then / l_ii */
            for (int64_t i = n - 1; i >= 0; i--) {
                for (int64_t k = i + 1; k < n; k++)
                    b[i] = psub(b[i], pmul(AT(A, lda, k, i), b[k]));
                b[i] = pdiv(b[i], AT(A, lda, i, i));
            }
        } else {
            /* U^T y = b: ascending dot form, then / u_ii */
            for (int64_t i = 0; i < n; i++) {
                for (int64_t k = 0; k < i; k++)
                    b[i] = psub(b[i], pmul(AT(A, lda, k, i), b[k]));
                b[i] = pdiv(b[i], AT(A, lda, i, i));
            }
            /* U x = y: i descending, k = n-1..i+1 descending, then / u_ii */
            for (int64_t i = n - 1; i >= 0; i--) {
                for (int64_t k = n - 1; k > i; k--)
                    b[i] = psub(b[i], pmul(AT(A, lda, i, k), b[k]));
                b[i] = pdiv(b[i], AT(A, lda, i, i));
            }
        }
    }
}
