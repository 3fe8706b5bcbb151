/*
 * posit_oracle.h -- plain CPU oracle for Posit(n,2) arithmetic and the
 * Posit(32,2) BLAS/LAPACK routines Rgemm, Rgetrf, Rpotrf, Rgetrs, Rpotrs.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library.  The CUDA
 * library never includes, links or calls it, and this file shares no code
 * with it.
 *
 * Words are passed as uint32_t bit patterns holding an n-bit posit in the
 * low n bits (n = 32 for every routine below that does not take `nbits`).
 * Matrices are column-major with a leading dimension, as in LAPACK.
 *
 * Paper: "Evaluation of POSIT Arithmetic with Accelerators", Sec. 2 (Eq. 1,
 * the format), Sec. 3 (Eq. GEMM_DEF, MPLAPACK Rgemm/Rgetrf/Rpotrf),
 * Sec. 5.1 (Rgetrs/Rpotrs for the error study).
 */
#ifndef POSIT_ORACLE_H
#define POSIT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- scalar Posit(nbits,2), 3 <= nbits <= 32 ---------------------------- */
uint32_t or_add(int nbits, uint32_t a, uint32_t b);
uint32_t or_sub(int nbits, uint32_t a, uint32_t b);
uint32_t or_mul(int nbits, uint32_t a, uint32_t b);
uint32_t or_div(int nbits, uint32_t a, uint32_t b);
uint32_t or_sqrt(int nbits, uint32_t a);
uint32_t or_neg(int nbits, uint32_t a);
uint32_t or_from_double(int nbits, double x);
double   or_to_double(int nbits, uint32_t p);
/* decode into sign, scale and fraction: returns 0 zero, 1 finite, 2 NaR;
   value = (-1)^neg * 2^scale * (1 + frac / 2^fbits)                        */
int      or_decode(int nbits, uint32_t p, int *neg, int *scale,
                   uint32_t *frac, int *fbits);

/* element-wise array forms (op: 0 add, 1 sub, 2 mul, 3 div, 4 sqrt) */
void or_elementwise(int nbits, int op, const uint32_t *a, const uint32_t *b,
                    uint32_t *out, int64_t count);
void or_from_double_array(int nbits, const double *x, uint32_t *out,
                          int64_t count);
void or_to_double_array(int nbits, const uint32_t *p, double *out,
                        int64_t count);

/* ---- Posit(32,2) BLAS / LAPACK (canonical operation order) -------------- */
void or_set_threads(int threads);
int  or_get_threads(void);

void or_rgemm(char transa, char transb, int64_t m, int64_t n, int64_t k,
              uint32_t alpha, const uint32_t *A, int64_t lda,
              const uint32_t *B, int64_t ldb, uint32_t beta,
              uint32_t *C, int64_t ldc);

/* unblocked LU with partial pivoting; ipiv 1-based; returns info */
int or_rgetrf(int64_t m, int64_t n, uint32_t *A, int64_t lda, int32_t *ipiv);
/* blocked right-looking LU (panel, row swaps, unit-lower trsm, Rgemm
   trailing update with alpha=-1, beta=1); same result for every nb */
int or_rgetrf_blocked(int64_t m, int64_t n, uint32_t *A, int64_t lda,
                      int32_t *ipiv, int64_t nb);
void or_rgetrs(char trans, int64_t n, int64_t nrhs, const uint32_t *A,
               int64_t lda, const int32_t *ipiv, uint32_t *B, int64_t ldb);

/* Cholesky, uplo 'L' (A = L L^T) or 'U' (A = U^T U); returns info */
int or_rpotrf(char uplo, int64_t n, uint32_t *A, int64_t lda);
int or_rpotrf_blocked(char uplo, int64_t n, uint32_t *A, int64_t lda,
                      int64_t nb);
void or_rpotrs(char uplo, int64_t n, int64_t nrhs, const uint32_t *A,
               int64_t lda, uint32_t *B, int64_t ldb);

#ifdef __cplusplus
}
#endif
#endif
