// internal.cuh -- helpers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/posit_gb300.h"
#include "posit_core.cuh"

namespace posit {

inline bool is_trans(char t) { return t == 'T' || t == 't' || t == 'C' || t == 'c'; }
inline bool is_notrans(char t) { return t == 'N' || t == 'n'; }
inline bool valid_trans(char t) { return is_trans(t) || is_notrans(t); }
inline bool is_lower(char u) { return u == 'L' || u == 'l'; }
inline bool is_upper(char u) { return u == 'U' || u == 'u'; }
__host__ __device__ inline int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }
__host__ __device__ inline int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Map the most recent launch error to the library's return code.
inline int launch_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? POSIT_OK : POSIT_ERR_CUDA;
}

// Triangle restriction of a C update: all, lower (i >= j) or upper (i <= j).
enum Tri { TRI_FULL = 0, TRI_LOWER = 1, TRI_UPPER = 2 };

// Rgemm without argument checking (used by the factorisations).
int rgemm_launch(bool ta, bool tb, int tri, int64_t m, int64_t n, int64_t k,
                 uint32_t alpha, const uint32_t *A, int64_t lda,
                 const uint32_t *B, int64_t ldb, uint32_t beta, uint32_t *C,
                 int64_t ldc, cudaStream_t stream);

// Same, skipped by the kernel when *abort_flag != 0 (read on the device).
int rgemm_launch_guarded(bool ta, bool tb, int tri, int64_t m, int64_t n, int64_t k,
                         uint32_t alpha, const uint32_t *A, int64_t lda,
                         const uint32_t *B, int64_t ldb, uint32_t beta, uint32_t *C,
                         int64_t ldc, const int32_t *abort_flag, cudaStream_t stream);

// Blocked factorisations on a caller-provided scratch block of
// getrf_scratch_bytes() / potrf_scratch_bytes() bytes (device memory).  With
// side != nullptr the next panel is factored on `side` while the trailing
// update runs on `stream` (lookahead; the same bits).
size_t getrf_scratch_bytes();
size_t potrf_scratch_bytes();
int getrf_run(int64_t m, int64_t n, uint32_t *A, int64_t lda, int32_t *ipiv, int32_t *info,
              void *scratch, cudaStream_t stream, cudaStream_t side = nullptr);
int potrf_run(bool upper, int64_t n, uint32_t *A, int64_t lda, int32_t *info, void *scratch,
              cudaStream_t stream, cudaStream_t side = nullptr);
// The library's lookahead stream on the current device (highest priority,
// created on first use, kept for the life of the process); nullptr on error.
cudaStream_t lookahead_stream();

// Solves on a caller-provided scratch block of scratch_bytes bytes (device
// memory); solve_scratch_bytes(n) is enough for any nrhs (smaller blocks
// solve fewer right-hand sides per launch, at least 8 n / 32 + 264 bytes).
size_t solve_scratch_bytes(int64_t n);
int getrs_run(bool trans, int64_t n, int64_t nrhs, const uint32_t *A, int64_t lda,
              const int32_t *ipiv, uint32_t *B, int64_t ldb, void *scratch, size_t scratch_bytes,
              cudaStream_t stream);
int potrs_run(bool upper, int64_t n, int64_t nrhs, const uint32_t *A, int64_t lda, uint32_t *B,
              int64_t ldb, void *scratch, size_t scratch_bytes, cudaStream_t stream);
// Same, skipped on the device when *abort_flag != 0 (a failed factorisation).
int potrs_run_guarded(bool upper, int64_t n, int64_t nrhs, const uint32_t *A, int64_t lda,
                      uint32_t *B, int64_t ldb, const int32_t *abort_flag, void *scratch,
                      size_t scratch_bytes, cudaStream_t stream);

// Batched factor + solve (batched.cu).
size_t batched_workspace_bytes(int max_n, int max_nrhs, const posit_plan &plan);
int batched_launch(const posit_problem *probs, const int32_t *order, int64_t count, int max_n,
                   int max_nrhs, const posit_plan &plan, void *workspace, cudaStream_t stream);

}  // namespace posit
