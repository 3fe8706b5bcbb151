/*
 * posit_gb300.h -- C ABI of the Posit(32,2) dense linear-algebra library for
 * GB300 (sm_103a).
 *
 * Paper: "Evaluation of POSIT Arithmetic with Accelerators" (HPC Asia 2024).
 *
 * Data.  A posit word is a uint32_t bit pattern of Posit(32,2) (Sec. 2, Eq. 1:
 * x = (-1)^s * 16^k * 2^e * 1.f).  0x00000000 is zero, 0x80000000 is NaR,
 * 0x40000000 is 1, negation is the two's complement of the word.  Matrices
 * are column-major: element (i, j) of X is X[i + j * ldX], ldX >= rows.
 *
 * Arithmetic.  Every multiply, add, divide and square root is rounded to
 * Posit(32,2) at once (round to nearest, ties to the even pattern, saturating
 * at minpos/maxpos, never to zero or NaR; NaR propagates; x/0 and sqrt(x<0)
 * are NaR).  There is no fused multiply-add and no wider accumulator, and the
 * order of the operations on every output element is fixed (documented per
 * routine), so results are bit-exact and independent of tiling or launch
 * shape.
 *
 * Memory and streams.  Every matrix, vector, pivot and info pointer is DEVICE
 * memory owned by the caller, unless a routine says otherwise.  Calls are
 * asynchronous and ordered on the CUDA stream `stream` (0 = legacy default
 * stream); outputs are valid after the stream reaches the call.  Where a
 * routine needs scratch memory it allocates it stream-ordered
 * (cudaMallocAsync) and frees it before returning; nothing outlives a call.
 *
 * Return value.  0 on success.  -i when argument i (1-based, in the order of
 * the signature) is invalid, as LAPACK's xerbla does, without aborting.
 * POSIT_ERR_* (below) for CUDA failures.  Numerical status (singular or not
 * positive definite matrices) is written to the device integer `info` with
 * LAPACK's meaning, never signalled through the return value.
 */
#ifndef POSIT_GB300_H
#define POSIT_GB300_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef uint32_t posit32_t;

#if defined(__GNUC__)
#define POSIT_API __attribute__((visibility("default")))
#else
#define POSIT_API
#endif

#define POSIT_OK 0
#define POSIT_ERR_CUDA (-1001)    /* a kernel launch or CUDA runtime call failed */
#define POSIT_ERR_ALLOC (-1002)   /* stream-ordered scratch allocation failed */
#define POSIT_ERR_TIMEOUT (-1003) /* a bounded device-side wait gave up */
#define POSIT_ERR_DEVICE (-1004)  /* no usable device */
#define POSIT_ERR_SCRATCH (-1005) /* posit_rgetrf_static: the fixed scratch is too small */

/* ---------------------------------------------------------------------------
 * Conversion and element-wise arithmetic (the paper's Add/Mul/Div/Sqrt
 * kernels, Sec. 4.2 / Table tabrandom: r[i] = p[i] op q[i]).
 * ------------------------------------------------------------------------ */

/* p[i] = posit nearest to x[i] (same rounding rule; NaN and +-Inf give NaR).
   x: count doubles, p: count words; both device memory.  -3 if count < 0. */
POSIT_API int posit_from_double(const double *x, posit32_t *p, int64_t count,
                      cudaStream_t stream);

/* x[i] = exact double value of p[i] (NaR gives a quiet NaN). */
POSIT_API int posit_to_double(const posit32_t *p, double *x, int64_t count,
                    cudaStream_t stream);

/* Element-wise op on count words: op 0 add (p+q), 1 sub (p-q), 2 mul (p*q),
   3 div (p/q), 4 sqrt (sqrt p; q is not read and may be NULL).
   -1 for an unknown op, -5 if count < 0. */
POSIT_API int posit_elementwise(int op, const posit32_t *p, const posit32_t *q,
                      posit32_t *r, int64_t count, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Rgemm: C = alpha op(A) op(B) + beta C            (Sec. 3, Eq. GEMM_DEF)
 *
 * op(X) = X for 'N'/'n', X^T for 'T'/'t' (and 'C'/'c').  op(A) is m x k,
 * op(B) is k x n, C is m x n.  lda >= max(1, rows of A as stored), likewise
 * ldb, ldc >= max(1, m).
 *
 * Order per element (the reference-BLAS loop order, every op rounded):
 *   c = (beta == 0) ? 0 : (beta == 1) ? C_ij : beta * C_ij
 *   for l = 0 .. k-1 ascending:  t = alpha * op(B)_lj ;  c = c + t * op(A)_il
 * beta == 0 means C is not read.  alpha == 0 or k == 0 gives C = beta C
 * without reading A or B.  m == 0 or n == 0 returns at once.
 * With alpha = -1 and beta = 1 this is the trailing-matrix update
 * C_ij <- C_ij - sum_l A_il B_lj of blocked LU and Cholesky (Sec. 4.4).
 * ------------------------------------------------------------------------ */
POSIT_API int posit_rgemm(char transa, char transb, int64_t m, int64_t n, int64_t k,
                posit32_t alpha, const posit32_t *A, int64_t lda,
                const posit32_t *B, int64_t ldb, posit32_t beta,
                posit32_t *C, int64_t ldc, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Rgetrf: LU factorisation with partial pivoting, A = P L U     (Sec. 3, the
 * LAPACK dgetrf the paper runs through MPLAPACK; Sec. 5.2)
 *
 * A: m x n (lda >= max(1, m)), overwritten by L (unit lower, below the
 * diagonal) and U.  ipiv: min(m, n) int32, 1-based: row i was swapped with
 * row ipiv[i] (LAPACK convention).  info: one device int32, set to 0, or to
 * j+1 for the first column j whose pivot is exactly zero (the factorisation
 * still completes; U is singular), or to POSIT_ERR_TIMEOUT if a bounded
 * device wait gave up.
 *
 * Order: for each column c in turn -- pivot = first row of largest |a_ic|
 * (i >= c) comparing the two's-complement absolute value of the words as
 * unsigned integers (so NaR ranks highest); swap rows c and pivot across all
 * columns; r = 1 / a_cc; l_ic = a_ic * r; a_ik = a_ik - l_ic * a_ck for all
 * i, k > c.  The blocked schedule (panels of up to 256 columns, trailing
 * update by Rgemm with alpha = -1, beta = 1) applies exactly these operations
 * to every element in the same order, so the result is bit-identical for
 * every block size.  Scratch: about 0.7 MB, stream-ordered.  The work is
 * issued on `stream` and, from the third panel on, on a library-owned
 * high-priority stream per device (created on the first call) that factors
 * the next panel while `stream` updates the trailing matrix; the two are
 * joined by events before the call returns, so the work is ordered on
 * `stream` as usual (also under stream capture).
 * Errors: -1 m < 0, -2 n < 0, -3 A NULL, -4 lda, -5 ipiv NULL, -6 info NULL.
 * ------------------------------------------------------------------------ */
POSIT_API int posit_rgetrf(int64_t m, int64_t n, posit32_t *A, int64_t lda, int32_t *ipiv,
                 int32_t *info, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Rgetrs: solve A X = B ('N') or A^T X = B ('T') with the factors of
 * posit_rgetrf (Sec. 5.1).  B: n x nrhs (ldb >= max(1, n)), overwritten by X.
 *
 * Order ('N'): the ipiv swaps for i = 0 .. n-1; then L y = b with y_i
 * receiving l_ij y_j for j = 0 .. i-1 ascending; then U x = y with x_i
 * receiving u_ik x_k for k = n-1 .. i+1 descending, then x_i = x_i / u_ii.
 * ('T'): U^T y = b, y_i receiving u_ki y_k for k ascending, then / u_ii;
 * L^T z = y, z_i receiving l_ki z_k for k = i+1 .. n-1 ascending (one serial
 * chain of n(n-1)/2 operations per column); the swaps in reverse order.
 * These are the reference-BLAS trsm orders.  No singularity check: x / 0 is
 * NaR.  Errors: -1 trans, -2 n, -3 nrhs, -4 A NULL, -5 lda, -6 ipiv NULL,
 * -7 B NULL, -8 ldb.  The environment variable POSIT_SOLVE_SMEM_LIMIT
 * (bytes), read at each call, caps the shared memory a solve kernel takes
 * per CTA (this and posit_rpotrs); columns that no longer fit are swapped
 * and solved by slower global-memory kernels, with the same results.
 * ------------------------------------------------------------------------ */
POSIT_API int posit_rgetrs(char trans, int64_t n, int64_t nrhs, const posit32_t *A, int64_t lda,
                 const int32_t *ipiv, posit32_t *B, int64_t ldb, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Rpotrf: Cholesky factorisation A = L L^T (uplo 'L') or U^T U ('U')
 * (Sec. 3, LAPACK dpotrf through MPLAPACK; Sec. 5.2).
 *
 * Only the uplo triangle of A (n x n, lda >= max(1, n)) is read and written.
 * Order (uplo 'L'): for each column j in turn -- d = a_jj; if d <= 0 or NaR:
 * info = j+1 and stop (a_jj keeps d); a_jj = sqrt(d); r = 1 / a_jj;
 * a_ij = a_ij * r (i > j); a_ik = a_ik - a_ij * a_kj for j < k <= i.  uplo
 * 'U' is the transposed mirror.  Blocked: panels of up to 256 columns, the
 * trailing triangle updated by Rgemm (alpha = -1, beta = 1); bit-identical
 * for every block size; the next panel is factored ahead on the library's
 * side stream as in posit_rgetrf.  After a failure (info > 0) columns
 * 0 .. info-2 hold their final values and the rest of the triangle is
 * unspecified.
 * Errors: -1 uplo, -2 n, -3 A NULL, -4 lda, -5 info NULL.
 * ------------------------------------------------------------------------ */
POSIT_API int posit_rpotrf(char uplo, int64_t n, posit32_t *A, int64_t lda, int32_t *info,
                 cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Rpotrs: solve A X = B with the factor of posit_rpotrf (Sec. 5.1).
 * Order (uplo 'L'): L y = b, y_i receiving l_ij y_j for j ascending, then
 * / l_ii; L^T x = y, x_i receiving l_ki x_k for k = i+1 .. n-1 ascending
 * (the reference trsm dot form; one serial chain of n(n-1)/2 operations per
 * column), then / l_ii.  (uplo 'U'): U^T y = b with k ascending then / u_ii;
 * U x = y with k descending then / u_ii.  Errors: -1 uplo, -2 n, -3 nrhs,
 * -4 A NULL, -5 lda, -6 B NULL, -7 ldb.
 * ------------------------------------------------------------------------ */
POSIT_API int posit_rpotrs(char uplo, int64_t n, int64_t nrhs, const posit32_t *A, int64_t lda,
                 posit32_t *B, int64_t ldb, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Batched factor + solve: many independent problems in one persistent launch
 * (the batching pattern built on the paper's Rgetrf/Rgetrs and
 * Rpotrf/Rpotrs, Sec. 5).
 *
 * problems: DEVICE array of `count` descriptors.  For each problem:
 *   kind POSIT_LU:       A (n x n, lda) is overwritten by its LU factors as
 *                        posit_rgetrf does, ipiv (n int32) receives the
 *                        pivots, B (n x nrhs, ldb) is overwritten by the
 *                        solution of A X = B as posit_rgetrs('N') gives it;
 *   kind POSIT_CHOLESKY: the lower triangle of A is overwritten by L as
 *                        posit_rpotrf('L') does and B by the posit_rpotrs('L')
 *                        solution (B is left unchanged if info > 0);
 *   kind POSIT_CHOLESKY_U: the same with the upper triangle, A = U^T U,
 *                        posit_rpotrf('U') and posit_rpotrs('U'), whose
 *                        solve has no serial chain.
 * *info (device int32, may be NULL) receives the factorisation's info.
 * Every output word equals the corresponding single-problem routine's.
 * order: optional DEVICE array (count int32): the problems are started in
 * this order (e.g. largest n first); NULL means 0, 1, 2, ...
 * max_n, max_nrhs: upper bounds over the problems (size the workspace).
 * plan: launch shape (any valid plan gives the same results):
 *   threads      threads per CTA (multiple of 32, <= 512)
 *   ctas_per_sm  persistent CTAs per SM
 *   smem_bytes   shared memory per CTA; a problem whose
 *                n*n + n*nrhs + n*max(nrhs, 1) decoded elements (8 bytes
 *                each) fit is kept there, others use the CTA's slice of
 *                the workspace.
 * workspace: DEVICE memory of posit_batched_workspace_size() bytes, or NULL
 * to allocate it stream-ordered inside the call.  With a workspace the call
 * performs no allocation and enqueues one memset and one kernel.
 * Errors: -1 count, -2 problems NULL, -4 max_n, -5 max_nrhs, -6 plan.
 * ------------------------------------------------------------------------ */
#define POSIT_LU 0
#define POSIT_CHOLESKY 1    /* uplo 'L' */
#define POSIT_CHOLESKY_U 2  /* uplo 'U' */

typedef struct posit_problem {
  int32_t kind;      /* POSIT_LU, POSIT_CHOLESKY or POSIT_CHOLESKY_U */
  int32_t n;
  int32_t nrhs;
  int32_t reserved;
  int64_t lda;
  int64_t ldb;
  posit32_t *A;
  posit32_t *B;
  int32_t *ipiv;     /* LU only */
  int32_t *info;
} posit_problem;

typedef struct posit_plan {
  int32_t threads;
  int32_t ctas_per_sm;
  int32_t smem_bytes;
  int32_t reserved;
} posit_plan;

/* Bytes of DEVICE workspace posit_factor_solve_batched needs for problems up
   to max_n x max_n with up to max_nrhs right-hand sides under `plan`
   (written to *bytes).  Errors: -1 max_n, -2 max_nrhs, -3 plan, -4 bytes. */
POSIT_API int posit_batched_workspace_size(int64_t max_n, int64_t max_nrhs,
                                           const posit_plan *plan, size_t *bytes);

/* The batched call described above. */
POSIT_API int posit_factor_solve_batched(int64_t count, const posit_problem *problems,
                                         const int32_t *order, int64_t max_n, int64_t max_nrhs,
                                         const posit_plan *plan, void *workspace,
                                         cudaStream_t stream);

/* Autotuner of the batched launch shape: times posit_factor_solve_batched on
 * `problems` (a DEVICE descriptor array, as above, with `order` as above)
 * under each of the `ncand` candidate plans in the HOST array `cands` and
 * writes the fastest to *best (HOST).  times_ms (HOST, ncand floats, or NULL)
 * receives each candidate's best time of `reps` runs, -1 for a plan that
 * could not be launched (e.g. more shared memory than an SM has).  Since
 * every plan computes the same bits, only time is compared; ties go to the
 * plan with fewer threads per SM.  The problems are not modified: the timed
 * runs work on device copies of A and B (stream-ordered allocations made and
 * freed inside the call).  Blocks until `stream` has finished.
 * Errors: -1 count (must be > 0), -2 problems NULL, -4 max_n, -5 max_nrhs,
 * -6 cands NULL or ncand < 1, -8 reps < 1, -9 best NULL; POSIT_ERR_ALLOC if
 * the copies do not fit; POSIT_ERR_CUDA if no candidate could be launched. */
POSIT_API int posit_autotune(int64_t count, const posit_problem *problems, const int32_t *order,
                             int64_t max_n, int64_t max_nrhs, const posit_plan *cands,
                             int32_t ncand, int32_t reps, posit_plan *best, float *times_ms,
                             cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Serving: a continuous-batching server for factor+solve requests (the
 * request-serving pattern over the paper's Rgetrf+Rgetrs / Rpotrf+Rpotrs).
 *
 * Requests carry HOST matrices (column-major, ld = n); the caller keeps A
 * and B readable until the request is admitted and X / info writable until
 * it completes (page-locked host memory lets the copies overlap).  Requests
 * are admitted in arrival order while their device state (A, B, pivots,
 * info) fits budget_bytes; it stays on the device until completion.  Requests
 * with n <= small_n_max are batched continuously: when the previous small
 * launch has finished, every admitted, not yet started small request (up to
 * max_batch) goes into one persistent posit_factor_solve_batched launch with
 * `plan`.  Larger requests run through the blocked multi-SM routines, up to
 * large_lanes of them at once on their own streams, concurrently with the
 * small lane.  Latency first: while a large lane is idle and no large
 * request waits, a waiting small request with n > batch_only_n_max takes
 * that lane (the multi-SM routines finish it sooner than one CTA of a
 * batch); under load the lanes are busy and such requests are batched
 * (batch_only_n_max >= small_n_max: every small request is batched).
 * X receives
 * the solution (LU: posit_rgetrs 'N'; Cholesky: posit_rpotrs 'L' or, for
 * POSIT_CHOLESKY_U, 'U' -- or B unchanged if the factorisation failed) and
 * *info the factorisation's info,
 * bit-identical to the single-request routines whatever the mix.
 *
 * The server is driven by its caller: posit_serve_poll retires finished
 * launches (non-blocking event queries), frees their memory, admits waiting
 * requests, starts launches on idle lanes, and returns the tags of the
 * requests completed since the previous poll.  Not thread-safe: one thread
 * drives one server.
 * ------------------------------------------------------------------------ */
typedef struct posit_serve_config {
  int64_t budget_bytes;  /* device memory for resident request state */
  int32_t small_n_max;   /* n <= this: batched lane */
  int32_t max_batch;     /* requests per batched launch */
  int32_t max_nrhs;      /* largest nrhs accepted */
  int32_t large_lanes;   /* concurrent large requests (streams); 0 means 16 */
  posit_plan plan;       /* batched launch shape */
  int32_t batch_only_n_max; /* small requests with n above this take an idle
                               large lane instead of waiting for a batch */
  int32_t reserved;
} posit_serve_config;

typedef struct posit_request {
  int32_t kind;          /* POSIT_LU, POSIT_CHOLESKY or POSIT_CHOLESKY_U */
  int32_t n;
  int32_t nrhs;
  int32_t reserved;
  const posit32_t *A;    /* HOST, n x n */
  const posit32_t *B;    /* HOST, n x nrhs */
  posit32_t *X;          /* HOST, n x nrhs, written at completion */
  int32_t *info;         /* HOST, written at completion */
  uint64_t tag;          /* returned by posit_serve_poll */
} posit_request;

typedef struct posit_serve_stats_t {
  int64_t pending;             /* submitted, waiting for memory */
  int64_t admitted;            /* total admitted */
  int64_t completed;           /* total completed */
  int64_t inflight_launches;
  int64_t launches;            /* total launches started */
  int64_t device_bytes_in_use;
  int64_t batched_requests;    /* requests that went through the small lane */
  int64_t largest_batch;       /* most requests in one small-lane launch */
} posit_serve_stats_t;

typedef struct posit_server posit_server;

/* Create a server (streams, batched workspace, staging).  Errors: -1 cfg,
   -2 out NULL, POSIT_ERR_ALLOC / POSIT_ERR_CUDA. */
POSIT_API int posit_serve_open(const posit_serve_config *cfg, posit_server **out);

/* Queue a request (copied; host pointers are used later, see above).
   Errors: -1 server NULL, -2 bad request (kind, sizes, NULL pointers, or a
   footprint larger than the whole budget). */
POSIT_API int posit_serve_submit(posit_server *server, const posit_request *req);

/* Make progress and collect up to max_done completed tags into done_tags
   (*n_done receives the count).  Never blocks on the GPU.
   Errors: -1 server NULL, -3 done_tags/max_done, -4 n_done NULL. */
POSIT_API int posit_serve_poll(posit_server *server, uint64_t *done_tags, int64_t max_done,
                               int64_t *n_done);

/* Counters of the server (host memory).  Errors: -1 server, -2 st NULL. */
POSIT_API int posit_serve_stats(const posit_server *server, posit_serve_stats_t *st);

/* Wait for the server's streams, free everything.  Errors: -1 server NULL. */
POSIT_API int posit_serve_close(posit_server *server);

/* ---------------------------------------------------------------------------
 * posit_selftest_wait: failure-detection self-test of the bounded device
 * waits.  (The paper has no counterpart; its factorisations never wait on
 * the device.)
 *
 * The panel kernels of posit_rgetrf / posit_rpotrf meet at grid barriers
 * whose waits give up after a time limit (2 s there), set an error flag,
 * write POSIT_ERR_TIMEOUT into info and return, instead of hanging the GPU.
 * This call runs that same barrier, with a limit of wait_ns nanoseconds, in
 * a state where it can never complete (two CTAs waiting for a third), so the
 * limit runs out: after the stream completes, *info (device int32) holds
 * POSIT_ERR_TIMEOUT and the context stays usable.  Asynchronous; takes
 * 256 bytes of stream-ordered scratch.
 * Errors: -1 wait_ns outside [1e3, 1e10], -2 info NULL, POSIT_ERR_ALLOC,
 * POSIT_ERR_CUDA.
 * ------------------------------------------------------------------------ */
POSIT_API int posit_selftest_wait(int64_t wait_ns, int32_t *info, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * posit_rgetrf_static: posit_rgetrf for callers that must not allocate.
 * (The paper has no counterpart; this is a library convenience.)
 *
 * Same arguments, results (bit for bit) and errors as posit_rgetrf, but the
 * routine makes no device allocation: its ~0.6 MB of scratch comes from a
 * fixed 1 MiB array compiled into the library, which every GPU that loads
 * the library keeps for the life of the process.  Meant for callers whose
 * device memory is fully held by another allocator, that run under strict
 * memory accounting, or that must not wait on an allocation.
 * - The first call on a device looks up the array's device address (once
 *   per device, with that device current); make that first call before any
 *   stream capture begins.
 * - All calls share the one array: calls whose work overlaps on the GPU
 *   (for example on two streams at once) race and give wrong results, so
 *   order them on one stream or synchronise between them.
 * - Returns POSIT_ERR_SCRATCH if the device would need more scratch than
 *   the array holds (devices with more than about 250 SMs).
 * ------------------------------------------------------------------------ */
POSIT_API int posit_rgetrf_static(int64_t m, int64_t n, posit32_t *A, int64_t lda,
                                  int32_t *ipiv, int32_t *info, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* POSIT_GB300_H */
