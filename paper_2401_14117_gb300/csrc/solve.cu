// solve.cu -- Rgetrs and Rpotrs (Sec. 5.1: the factors solve A x = b for the
// error study), in the reference-BLAS trsm operation orders that LAPACK's
// dgetrs/dpotrs (and MPLAPACK's R versions) use.
//
// Two kinds of triangular solve occur:
//   * "wavefront": every unknown receives its updates in the order in which
//     the unknowns are solved -- forward with ascending k, or backward with
//     descending k (column-oriented trsm; also the dot-form forward solve with
//     ascending k).  trsv_wave_kernel solves 64-row blocks one after another;
//     after each block is solved (by the CTA that owns it) and published, every
//     CTA applies that block's unknowns to its own later rows.  One bounded
//     grid barrier per block.
//   * "dot-form backward": x_i = (b_i - sum_{k = i+1 .. n-1, ascending}
//     a_ki x_k) / a_ii, i descending (reference trsm Left-Lower-Transpose).
//     x_i's first subtraction needs x_{i+1}, the last unknown to finish, so
//     the n(n-1)/2 subtractions form one serial chain per right-hand side.
//     trsv_dot_backward_kernel computes the products of each row in parallel
//     and runs the chain of rounded subtractions in one thread.
//
// Row swaps (ipiv, LAPACK convention) are applied by a one-CTA-per-column
// kernel on a shared-memory copy of the column.
#include "internal.cuh"

namespace posit {
namespace {

constexpr int ST = 256;        // threads per CTA
constexpr int WBS = 64;        // wavefront block size
constexpr int NRHS_CHUNK = 8;  // right-hand sides per wavefront launch
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool solve_barrier(unsigned *bar, unsigned nblocks, int *err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = bar + 1;
    unsigned gen = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long t0 = global_ns();
      while (*vgen == gen) {
        if (*(volatile int *)err) break;
        if (global_ns() - t0 > kWaitNs) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int *)err == 0;
}

struct TriArgs {
  const uint32_t *A;
  int64_t lda;
  uint32_t *B;
  int64_t ldb;
  int64_t n;
  int nrhs;
  int trans;     // element (i, k) of the triangle at A[k + i*lda] instead of A[i + k*lda]
  int backward;  // solve order: 0 ascending, 1 descending
  int unit;      // unit diagonal (no division)
  int nblk;      // number of WBS-row blocks
  int bpc;       // blocks per CTA
  unsigned *bar;
  int *err;
  const int32_t *abort_flag;  // skip the solve when *abort_flag != 0
};

__device__ __forceinline__ uint32_t tri_at(const TriArgs &a, int64_t i, int64_t k) {
  return a.trans ? a.A[k + i * a.lda] : a.A[i + k * a.lda];
}

// rows [r0, r1) of block b (block index in solve order J maps to b)
__device__ __forceinline__ int64_t block_row0(const TriArgs &a, int J) {
  int b = a.backward ? (a.nblk - 1 - J) : J;
  return (int64_t)b * WBS;
}

__global__ void __launch_bounds__(ST, 1) trsv_wave_kernel(TriArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nrhs = a.nrhs;
  pz *xs = reinterpret_cast<pz *>(smem_raw);            // [bpc*WBS][nrhs] own rows
  pz *xj = xs + (size_t)a.bpc * WBS * nrhs;              // [WBS][nrhs] published block
  pz *at = xj + (size_t)WBS * nrhs;                      // [WBS][WBS] tile of A
  const int tid = threadIdx.x;
  const int g = blockIdx.x;
  const unsigned G = gridDim.x;
  const int J0 = g * a.bpc, J1 = min(a.nblk, (g + 1) * a.bpc);
  if (a.abort_flag && *(volatile const int32_t *)a.abort_flag != 0) return;  // all CTAs alike

  // load own rows of B
  for (int J = J0; J < J1; ++J) {
    int64_t r0 = block_row0(a, J);
    int nr = (int)min64(WBS, a.n - r0);
    for (int idx = tid; idx < WBS * nrhs; idx += ST) {
      int r = idx % WBS, c = idx / WBS;
      pz v = pz_zero();
      if (r < nr) v = pz_decode(a.B[(r0 + r) + c * a.ldb]);
      xs[((size_t)(J - J0) * WBS + r) * nrhs + c] = v;
    }
  }
  __syncthreads();

  for (int J = 0; J < a.nblk; ++J) {
    const int64_t r0 = block_row0(a, J);
    const int nr = (int)min64(WBS, a.n - r0);
    if (J >= J0 && J < J1) {
      // the diagonal tile, decoded into shared memory in one pass:
      // at[r][t] = a(r0 + r, r0 + t)
      for (int idx = tid; idx < WBS * WBS; idx += ST) {
        int r, t;
        if (a.trans) { t = idx % WBS; r = idx / WBS; } else { r = idx % WBS; t = idx / WBS; }
        pz v = pz_zero();
        if (r < nr && t < nr) v = pz_decode(tri_at(a, r0 + r, r0 + t));
        at[r * WBS + t] = v;
      }
      __syncthreads();
      // solve the diagonal block in solve order
      pz *xb = xs + (size_t)(J - J0) * WBS * nrhs;
      for (int s = 0; s < nr; ++s) {
        const int t = a.backward ? (nr - 1 - s) : s;
        for (int c = tid; c < nrhs; c += ST) {
          pz x = xb[t * nrhs + c];
          if (!a.unit) x = pz_div(x, at[t * WBS + t]);
          xb[t * nrhs + c] = x;
          a.B[(r0 + t) + c * a.ldb] = pz_to_bits(x);
        }
        __syncthreads();
        const int nlater = nr - 1 - s;  // rows after t in solve order
        for (int idx = tid; idx < nlater * nrhs; idx += ST) {
          int q = idx / nrhs, c = idx % nrhs;
          int r = a.backward ? (t - 1 - q) : (t + 1 + q);
          pz *x = &xb[r * nrhs + c];
          *x = pz_sub(*x, pz_mul(at[r * WBS + t], xb[t * nrhs + c]));
        }
        __syncthreads();
      }
    }
    if (!solve_barrier(a.bar, G, a.err)) return;
    // apply block J to the own blocks that come later in solve order
    bool any = J1 > max(J0, J + 1);
    if (!any) continue;
    for (int idx = tid; idx < nr * nrhs; idx += ST) {
      int r = idx % nr, c = idx / nr;
      uint32_t w = __ldcg(&a.B[(r0 + r) + c * a.ldb]);
      xj[r * nrhs + c] = pz_decode(w);
    }
    for (int J2 = max(J0, J + 1); J2 < J1; ++J2) {
      const int64_t q0 = block_row0(a, J2);
      const int nq = (int)min64(WBS, a.n - q0);
      __syncthreads();
      // tile at[r][t] = a(q0 + r, r0 + t), loaded along the contiguous index
      for (int idx = tid; idx < WBS * WBS; idx += ST) {
        int r, t;
        if (a.trans) { t = idx % WBS; r = idx / WBS; } else { r = idx % WBS; t = idx / WBS; }
        pz v = pz_zero();
        if (r < nq && t < nr) v = pz_decode(tri_at(a, q0 + r, r0 + t));
        at[r * WBS + t] = v;
      }
      __syncthreads();
      pz *xq = xs + (size_t)(J2 - J0) * WBS * nrhs;
      for (int idx = tid; idx < nq * nrhs; idx += ST) {
        int r = idx % nq, c = idx / nq;
        pz acc = xq[r * nrhs + c];
        for (int s = 0; s < nr; ++s) {
          int t = a.backward ? (nr - 1 - s) : s;
          acc = pz_sub(acc, pz_mul(at[r * WBS + t], xj[t * nrhs + c]));
        }
        xq[r * nrhs + c] = acc;
      }
    }
    __syncthreads();
  }
}

// x_i = (b_i - sum_{k>i, ascending} a(k, i) x_k) / a(i, i), i = n-1 .. 0,
// for one right-hand side per CTA (column blockIdx.x of B).  a(k, i) is
// A[k + i*lda] (column i below the diagonal).  The products of a row are
// formed in parallel (the next chunk while the current one is consumed) and
// stored negated; one thread runs the chain of rounded additions, the only
// serial part, with the short-path addition pz_add_serial (a NaR product or
// b_i makes x_i NaR; that test is off the chain's dependency path).
__global__ void __launch_bounds__(ST) trsv_dot_backward_kernel(const uint32_t *__restrict__ A,
                                                                int64_t lda, uint32_t *B,
                                                                int64_t ldb, int64_t n, int unit,
                                                                const int32_t *abort_flag) {
  __shared__ pz prod[2][ST + 1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pz *x = reinterpret_cast<pz *>(smem_raw);  // [n] the right-hand side / solution
  uint32_t *b = B + (int64_t)blockIdx.x * ldb;
  const int tid = threadIdx.x;
  if (abort_flag && *abort_flag != 0) return;
  for (int64_t i = tid; i < n; i += ST) x[i] = pz_decode(b[i]);
  __syncthreads();
  for (int64_t i = n - 1; i >= 0; --i) {
    const uint32_t *col = A + i * lda;
    {
      int64_t k = i + 1 + tid;
      if (k < n) {
        pz p = pz_mul(pz_decode(col[k]), x[k]);
        prod[0][tid] = pz{p.s, p.m ^ 0x80000000u};
      }
    }
    __syncthreads();
    pz acc = x[i];
    bool nar = pz_is_nar(acc);
    int buf = 0;
    for (int64_t k0 = i + 1; k0 < n; k0 += ST) {
      int64_t kn = k0 + ST + tid;
      if (kn < n) {
        pz p = pz_mul(pz_decode(col[kn]), x[kn]);
        prod[buf ^ 1][tid] = pz{p.s, p.m ^ 0x80000000u};
      }
      if (tid == 0) {
        const int cnt = (int)min64(ST, n - k0);
        const pz *pr = prod[buf];
        pz pn = pr[0];
#pragma unroll 4
        for (int t = 0; t < cnt; ++t) {
          const pz p = pn;
          pn = pr[t + 1];  // next link's product, loaded ahead (row padded by one)
          nar |= p.s >= PZ_NAR_T;
          acc = pz_add_serial(acc, p);
        }
      }
      __syncthreads();
      buf ^= 1;
    }
    if (tid == 0) {
      pz v = nar ? pz_nar() : pz_canon(acc, false);
      if (!unit) v = pz_div(v, pz_decode(col[i]));
      x[i] = v;
    }
    __syncthreads();
  }
  for (int64_t i = tid; i < n; i += ST) b[i] = pz_to_bits(x[i]);
}

// LAPACK row swaps on each column of B: forward (i = 0 .. n-1) or reverse.
__global__ void __launch_bounds__(ST) laswp_vec_kernel(uint32_t *B, int64_t ldb, int64_t n,
                                                       const int32_t *__restrict__ ipiv,
                                                       int reverse) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t *v = reinterpret_cast<uint32_t *>(smem_raw);
  uint32_t *b = B + (int64_t)blockIdx.x * ldb;
  for (int64_t i = threadIdx.x; i < n; i += ST) v[i] = b[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int64_t s = 0; s < n; ++s) {
      int64_t i = reverse ? (n - 1 - s) : s;
      int64_t p = ipiv[i] - 1;
      uint32_t t = v[i];
      v[i] = v[p];
      v[p] = t;
    }
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += ST) b[i] = v[i];
}

// same, directly in global memory (columns too long for shared memory)
__global__ void laswp_vec_global_kernel(uint32_t *B, int64_t ldb, int64_t n,
                                        const int32_t *__restrict__ ipiv, int reverse) {
  if (threadIdx.x != 0) return;
  uint32_t *b = B + (int64_t)blockIdx.x * ldb;
  for (int64_t s = 0; s < n; ++s) {
    int64_t i = reverse ? (n - 1 - s) : s;
    int64_t p = ipiv[i] - 1;
    uint32_t t = b[i];
    b[i] = b[p];
    b[p] = t;
  }
}

__global__ void trsv_dot_backward_global_kernel(const uint32_t *__restrict__ A, int64_t lda,
                                                uint32_t *B, int64_t ldb, int64_t n, int unit,
                                                const int32_t *abort_flag) {
  // columns too long for shared memory: one thread per right-hand side
  if (threadIdx.x != 0) return;
  if (abort_flag && *abort_flag != 0) return;
  uint32_t *b = B + (int64_t)blockIdx.x * ldb;
  for (int64_t i = n - 1; i >= 0; --i) {
    const uint32_t *col = A + i * lda;
    pz acc = pz_decode(b[i]);
    for (int64_t k = i + 1; k < n; ++k) acc = pz_sub(acc, pz_mul(pz_decode(col[k]), pz_decode(b[k])));
    if (!unit) acc = pz_div(acc, pz_decode(col[i]));
    b[i] = pz_to_bits(acc);
  }
}

struct Limits {
  int sms, smem_optin;
};

int limits(Limits &l) {
  int dev;
  if (cudaGetDevice(&dev) != cudaSuccess) return POSIT_ERR_DEVICE;
  if (cudaDeviceGetAttribute(&l.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return POSIT_ERR_DEVICE;
  if (cudaDeviceGetAttribute(&l.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
      cudaSuccess)
    return POSIT_ERR_DEVICE;
  return POSIT_OK;
}

int laswp_vec(uint32_t *B, int64_t ldb, int64_t n, int64_t nrhs, const int32_t *ipiv,
              bool reverse, const Limits &l, cudaStream_t stream) {
  size_t smem = (size_t)n * 4;
  if (smem + 1024 <= (size_t)l.smem_optin) {
    if (cudaFuncSetAttribute(laswp_vec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return POSIT_ERR_CUDA;
    laswp_vec_kernel<<<(unsigned)nrhs, ST, smem, stream>>>(B, ldb, n, ipiv, reverse);
  } else {
    laswp_vec_global_kernel<<<(unsigned)nrhs, 32, 0, stream>>>(B, ldb, n, ipiv, reverse);
  }
  return launch_status();
}

// scratch for the wavefront barrier: 2 unsigned + 1 int
constexpr size_t kWaveScratch = 256;

int trsv_wave(const uint32_t *A, int64_t lda, int trans, int backward, int unit, uint32_t *B,
              int64_t ldb, int64_t n, int64_t nrhs, void *scratch, const Limits &l,
              cudaStream_t stream, const int32_t *abort_flag = nullptr) {
  const int nblk = (int)ceil_div(n, WBS);
  for (int64_t c0 = 0; c0 < nrhs; c0 += NRHS_CHUNK) {
    const int nr = (int)min64(NRHS_CHUNK, nrhs - c0);
    int G = (int)min64(l.sms, nblk);
    int bpc = (int)ceil_div(nblk, G);
    G = (int)ceil_div(nblk, bpc);
    size_t smem = ((size_t)bpc * WBS * nr + (size_t)WBS * nr + (size_t)WBS * WBS) * sizeof(pz);
    if (smem + 1024 > (size_t)l.smem_optin) return POSIT_ERR_DEVICE;  // n beyond ~1.8M rows
    if (cudaMemsetAsync(scratch, 0, kWaveScratch, stream) != cudaSuccess) return POSIT_ERR_CUDA;
    if (cudaFuncSetAttribute(trsv_wave_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return POSIT_ERR_CUDA;
    TriArgs ta;
    ta.A = A; ta.lda = lda; ta.B = B + c0 * ldb; ta.ldb = ldb; ta.n = n; ta.nrhs = nr;
    ta.trans = trans; ta.backward = backward; ta.unit = unit; ta.nblk = nblk; ta.bpc = bpc;
    ta.bar = static_cast<unsigned *>(scratch);
    ta.err = reinterpret_cast<int *>(static_cast<char *>(scratch) + 2 * sizeof(unsigned));
    ta.abort_flag = abort_flag;
    void *args[] = {&ta};
    if (cudaLaunchCooperativeKernel((const void *)trsv_wave_kernel, dim3(G), dim3(ST), args, smem,
                                    stream) != cudaSuccess)
      return POSIT_ERR_CUDA;
  }
  return POSIT_OK;
}

int trsv_dot_backward(const uint32_t *A, int64_t lda, int unit, uint32_t *B, int64_t ldb,
                      int64_t n, int64_t nrhs, const Limits &l, cudaStream_t stream,
                      const int32_t *abort_flag = nullptr) {
  size_t smem = (size_t)n * sizeof(pz);
  if (smem + 4096 <= (size_t)l.smem_optin) {
    if (cudaFuncSetAttribute(trsv_dot_backward_kernel,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return POSIT_ERR_CUDA;
    trsv_dot_backward_kernel<<<(unsigned)nrhs, ST, smem, stream>>>(A, lda, B, ldb, n, unit,
                                                                   abort_flag);
  } else {
    trsv_dot_backward_global_kernel<<<(unsigned)nrhs, 32, 0, stream>>>(A, lda, B, ldb, n, unit,
                                                                       abort_flag);
  }
  return launch_status();
}

}  // namespace

size_t solve_scratch_bytes() { return kWaveScratch; }

int getrs_run(bool trans, int64_t n, int64_t nrhs, const uint32_t *A, int64_t lda,
              const int32_t *ipiv, uint32_t *B, int64_t ldb, void *scratch, cudaStream_t stream) {
  Limits l;
  int st = limits(l);
  if (st) return st;
  if (!trans) {
    if ((st = laswp_vec(B, ldb, n, nrhs, ipiv, false, l, stream))) return st;
    // L y = b (unit lower): ascending, column order
    if ((st = trsv_wave(A, lda, 0, 0, 1, B, ldb, n, nrhs, scratch, l, stream))) return st;
    // U x = y: descending, column order, divide by u_ii
    return trsv_wave(A, lda, 0, 1, 0, B, ldb, n, nrhs, scratch, l, stream);
  }
  // U^T y = b: ascending dot form (a wavefront over U accessed transposed)
  if ((st = trsv_wave(A, lda, 1, 0, 0, B, ldb, n, nrhs, scratch, l, stream))) return st;
  // L^T z = y, unit: dot form, k ascending -- serial chain
  if ((st = trsv_dot_backward(A, lda, 1, B, ldb, n, nrhs, l, stream))) return st;
  return laswp_vec(B, ldb, n, nrhs, ipiv, true, l, stream);
}

int potrs_run_guarded(bool upper, int64_t n, int64_t nrhs, const uint32_t *A, int64_t lda,
                      uint32_t *B, int64_t ldb, const int32_t *abort_flag, void *scratch,
                      cudaStream_t stream) {
  Limits l;
  int st = limits(l);
  if (st) return st;
  if (!upper) {
    // L y = b: ascending, then divide
    if ((st = trsv_wave(A, lda, 0, 0, 0, B, ldb, n, nrhs, scratch, l, stream, abort_flag)))
      return st;
    // L^T x = y: dot form, k ascending -- serial chain
    return trsv_dot_backward(A, lda, 0, B, ldb, n, nrhs, l, stream, abort_flag);
  }
  // U^T y = b: ascending dot form
  if ((st = trsv_wave(A, lda, 1, 0, 0, B, ldb, n, nrhs, scratch, l, stream, abort_flag)))
    return st;
  // U x = y: descending, column order
  return trsv_wave(A, lda, 0, 1, 0, B, ldb, n, nrhs, scratch, l, stream, abort_flag);
}

int potrs_run(bool upper, int64_t n, int64_t nrhs, const uint32_t *A, int64_t lda, uint32_t *B,
              int64_t ldb, void *scratch, cudaStream_t stream) {
  return potrs_run_guarded(upper, n, nrhs, A, lda, B, ldb, nullptr, scratch, stream);
}

}  // namespace posit

using namespace posit;

extern "C" int posit_rgetrs(char trans, int64_t n, int64_t nrhs, const posit32_t *A, int64_t lda,
                            const int32_t *ipiv, posit32_t *B, int64_t ldb, cudaStream_t stream) {
  if (!valid_trans(trans)) return -1;
  if (n < 0) return -2;
  if (nrhs < 0) return -3;
  if (lda < max64(1, n)) return -5;
  if (ldb < max64(1, n)) return -8;
  if (n == 0 || nrhs == 0) return POSIT_OK;
  if (!A) return -4;
  if (!ipiv) return -6;
  if (!B) return -7;
  void *scratch = nullptr;
  if (cudaMallocAsync(&scratch, solve_scratch_bytes(), stream) != cudaSuccess) {
    cudaGetLastError();
    return POSIT_ERR_ALLOC;
  }
  int st = getrs_run(is_trans(trans), n, nrhs, A, lda, ipiv, B, ldb, scratch, stream);
  cudaFreeAsync(scratch, stream);
  return st;
}

extern "C" int posit_rpotrs(char uplo, int64_t n, int64_t nrhs, const posit32_t *A, int64_t lda,
                            posit32_t *B, int64_t ldb, cudaStream_t stream) {
  if (!is_lower(uplo) && !is_upper(uplo)) return -1;
  if (n < 0) return -2;
  if (nrhs < 0) return -3;
  if (lda < max64(1, n)) return -5;
  if (ldb < max64(1, n)) return -7;
  if (n == 0 || nrhs == 0) return POSIT_OK;
  if (!A) return -4;
  if (!B) return -6;
  void *scratch = nullptr;
  if (cudaMallocAsync(&scratch, solve_scratch_bytes(), stream) != cudaSuccess) {
    cudaGetLastError();
    return POSIT_ERR_ALLOC;
  }
  int st = potrs_run(is_upper(uplo), n, nrhs, A, lda, B, ldb, scratch, stream);
  cudaFreeAsync(scratch, stream);
  return st;
}
