// factor.cu -- blocked right-looking Rgetrf (LU with partial pivoting) and
// Rpotrf (Cholesky) on the GPU (Sec. 3: LAPACK dgetrf/dpotrf structure with
// Rgemm as the trailing-matrix update; Sec. 5.2 runs them with only Rgemm
// offloaded -- here every step runs on the device and the host only enqueues).
//
// Per panel of jb columns starting at column j:
//   LU:   panel_kernel (LU)  pivot search, row swap inside the panel, scaling by
//                            r = 1 / pivot, rank-1 updates of the panel columns
//         laswp_kernel       the panel's swaps on the columns left and right
//         trsm_llu_kernel    U12 <- L11^-1 A12 (unit lower, forward)
//         rgemm              A22 <- A22 - L21 U12   (alpha = -1, beta = 1)
//   Chol: panel_kernel (Chol) sqrt of the diagonal, scaling by its reciprocal,
//                            updates of the panel's lower triangle (this also
//                            performs the trsm of the rows below the block)
//         rgemm (lower)      A22 <- A22 - L21 L21^T on the lower triangle
//
// Every element receives its updates in ascending column order, one rounded
// multiply and one rounded subtract each, exactly as the unblocked algorithm
// does, so the result is the same for every jb.  From the third panel on the
// next panel is factored on a second stream while the rest of the trailing
// update runs (lookahead, getrf_run / potrf_run); the order per element is
// unchanged.
//
// The panel kernel is a cooperative launch: G CTAs own contiguous chunks of
// the panel's rows, kept decoded in shared memory for the whole panel, and
// meet at one grid barrier per column.  The barrier's wait is bounded (about
// 2 s of global time); a CTA that gives up sets the error flag, writes
// POSIT_ERR_TIMEOUT into info, and every CTA returns.
#include <cooperative_groups.h>

#include <mutex>

#include "internal.cuh"

namespace posit {
namespace {

constexpr int PT = 256;           // panel kernel threads
constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded barrier wait

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier over `nblocks` co-resident CTAs (cooperative launch).  bar[0]
// is a counter of arrivals that only grows (the host zeroes it before each
// launch): the CTA whose arrival returns `old` waits until the counter
// reaches the next multiple of nblocks.  One atomic per CTA and a spin on an
// acquire load; the error flag and the clock are looked at every 256 polls,
// and the wait gives up after wait_ns of global time (2 s in the
// factorisations).  Returns false after a timeout (or another CTA's).
__device__ bool grid_barrier(unsigned *bar, unsigned nblocks, int *err, int32_t *info,
                             unsigned long long wait_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned old = atomicAdd(bar, 1u);
    const unsigned target = (old / nblocks + 1u) * nblocks;
    unsigned long long t0 = 0;
    unsigned polls = 0;
    while ((int)(ld_acquire(bar) - target) < 0) {
      if ((++polls & 255u) == 0u) {
        if (*(volatile int *)err) break;
        const unsigned long long now = global_ns();
        if (t0 == 0) {
          t0 = now;
        } else if (now - t0 > wait_ns) {
          atomicExch(err, 1);
          atomicExch(info, POSIT_ERR_TIMEOUT);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int *)err == 0;
}

// |x| ordering key of a decoded value: (scale, magnitude) lexicographic, which
// is the order of the words' two's-complement absolute values (NaR largest,
// zero smallest).
__device__ __forceinline__ uint64_t abs_key(pz a) {
  if (pz_is_nar(a)) return ~0ull;
  if (pz_is_zero(a)) return 1ull;  // 0 is kept for "no candidate"
  return ((uint64_t)(uint32_t)(a.s + (1 << 24)) << 32) | (uint64_t)(a.m & 0x7FFFFFFFu);
}

struct PanelArgs {
  uint32_t *A;
  int64_t lda;
  int64_t m;     // rows of the matrix (the panel covers rows j .. m-1)
  int64_t j;     // first column (and first row) of the panel
  int jb;        // panel width
  int R;         // rows per CTA
  int trans;     // element (i, k) at A[k + i*lda] (Cholesky, upper storage)
  int chol;      // 0: LU with partial pivoting, 1: Cholesky
  int32_t *ipiv;
  int32_t *info;
  // scratch (zeroed before the first panel)
  unsigned *bar;
  int *err;
  uint64_t *cand_key;   // [2][G]
  int64_t *cand_row;    // [2][G]
  pz *cand_vals;        // [2][G][jb]
  pz *xrow;             // LU: old pivot row [2][jb]; Chol: broadcast column [2][jb]
  pz *diag;             // Chol: next diagonal value [2]
};

__device__ __forceinline__ int64_t panel_addr(const PanelArgs &a, int64_t i, int64_t k) {
  return a.trans ? (k + i * a.lda) : (i + k * a.lda);
}

__global__ void __launch_bounds__(PT, 1) panel_kernel(PanelArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int jb = a.jb, R = a.R;
  pz *tile = reinterpret_cast<pz *>(smem_raw);  // [R][jb]
  pz *prow = tile + (size_t)R * jb;             // [jb]
  __shared__ uint64_t red_key[PT / 32];
  __shared__ int64_t red_row[PT / 32];
  __shared__ pz s_r;   // reciprocal of the pivot / of the diagonal sqrt
  __shared__ int s_flag;
  __shared__ int64_t s_piv;

  const int tid = threadIdx.x;
  const int g = blockIdx.x;
  const unsigned G = gridDim.x;
  const int64_t row0 = a.j + (int64_t)g * R;            // first global row of this CTA
  const int nrows = (int)max64(0, min64((int64_t)R, a.m - row0));

  if (a.chol && *(volatile int32_t *)a.info != 0) return;  // an earlier panel failed

  // load this CTA's rows of the panel, decoded
  for (int idx = tid; idx < R * jb; idx += PT) {
    int r, c;
    if (a.trans) { c = idx % jb; r = idx / jb; } else { r = idx % R; c = idx / R; }
    pz v = pz_zero();
    if (r < nrows) v = pz_decode(a.A[panel_addr(a, row0 + r, a.j + c)]);
    tile[(size_t)r * jb + c] = v;
  }
  __syncthreads();

  if (a.chol) {
    // diagonal value of column 0, published by the CTA owning row j
    if (g == 0 && tid == 0) a.diag[0] = tile[0];
    if (!grid_barrier(a.bar, G, a.err, a.info, kWaitNs)) return;
  }

  for (int c = 0; c < jb; ++c) {
    const int buf = c & 1;
    const int64_t gcol = a.j + c;            // global column, = global pivot row
    const int owner_c = (int)(c / R);        // CTA holding row gcol
    const int lrow_c = c - owner_c * R;      // its local index there

    if (!a.chol) {
      // ---------------- LU: pivot search ------------------------------------
      uint64_t best = 0;
      int64_t brow = INT64_MAX;
      for (int r = tid; r < nrows; r += PT) {
        int64_t gr = row0 + r;
        if (gr < gcol) continue;
        uint64_t k = abs_key(tile[(size_t)r * jb + c]);
        if (k > best || (k == best && gr < brow)) { best = k; brow = gr; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        uint64_t ok = __shfl_down_sync(0xFFFFFFFFu, best, off);
        int64_t orow = __shfl_down_sync(0xFFFFFFFFu, brow, off);
        if (ok > best || (ok == best && orow < brow)) { best = ok; brow = orow; }
      }
      if ((tid & 31) == 0) { red_key[tid >> 5] = best; red_row[tid >> 5] = brow; }
      __syncthreads();
      if (tid == 0) {
        for (int w = 1; w < PT / 32; ++w)
          if (red_key[w] > best || (red_key[w] == best && red_row[w] < brow)) {
            best = red_key[w];
            brow = red_row[w];
          }
        __stcg(&a.cand_key[buf * G + g], best);
        __stcg(&a.cand_row[buf * G + g], brow);
        s_piv = brow;
      }
      __syncthreads();
      // the candidate row's panel values, and the current row gcol
      if (s_piv != INT64_MAX) {
        int lr = (int)(s_piv - row0);
        pz *dst = a.cand_vals + ((size_t)buf * G + g) * jb;
        for (int k = tid; k < jb; k += PT) dst[k] = tile[(size_t)lr * jb + k];
      }
      if (g == owner_c) {
        pz *dst = a.xrow + (size_t)buf * jb;
        for (int k = tid; k < jb; k += PT) dst[k] = tile[(size_t)lrow_c * jb + k];
      }
      if (!grid_barrier(a.bar, G, a.err, a.info, kWaitNs)) return;

      // every CTA picks the same pivot: largest |a|, then the lowest row
      // (candidates read in parallel, then a warp / block reduction)
      {
        uint64_t bk = 0;
        int64_t br = INT64_MAX;
        for (unsigned w = tid; w < G; w += PT) {
          uint64_t k = __ldcg(&a.cand_key[buf * G + w]);
          int64_t r = __ldcg(&a.cand_row[buf * G + w]);
          if (r != INT64_MAX && (k > bk || (k == bk && r < br))) { bk = k; br = r; }
        }
        for (int off = 16; off > 0; off >>= 1) {
          uint64_t ok = __shfl_down_sync(0xFFFFFFFFu, bk, off);
          int64_t orow = __shfl_down_sync(0xFFFFFFFFu, br, off);
          if (ok > bk || (ok == bk && orow < br)) { bk = ok; br = orow; }
        }
        if ((tid & 31) == 0) { red_key[tid >> 5] = bk; red_row[tid >> 5] = br; }
        __syncthreads();
        if (tid == 0) {
          for (int w = 1; w < PT / 32; ++w)
            if (red_key[w] > bk || (red_key[w] == bk && red_row[w] < br)) {
              bk = red_key[w];
              br = red_row[w];
            }
          s_piv = br;
          // the winning CTA is the one whose rows contain br
          s_flag = (int)((br - a.j) / a.R);
        }
        __syncthreads();
      }
      const int64_t p = s_piv;
      const pz *pv = a.cand_vals + ((size_t)buf * G + s_flag) * jb;
      for (int k = tid; k < jb; k += PT) {
        pz v;
        v.s = __ldcg(&pv[k].s);
        v.m = __ldcg(&pv[k].m);
        prow[k] = v;
      }
      __syncthreads();
      const bool zero = pz_is_zero(prow[c]);
      if (!zero && p != gcol) {
        if (g == owner_c)
          for (int k = tid; k < jb; k += PT) tile[(size_t)lrow_c * jb + k] = prow[k];
        if (p >= row0 && p < row0 + nrows) {
          const pz *old = a.xrow + (size_t)buf * jb;
          int lr = (int)(p - row0);
          for (int k = tid; k < jb; k += PT) {
            pz v;
            v.s = __ldcg(&old[k].s);
            v.m = __ldcg(&old[k].m);
            tile[(size_t)lr * jb + k] = v;
          }
        }
      }
      if (tid == 0) {
        if (!zero) s_r = pz_div(pz_one(), prow[c]);
        if (g == 0) {
          a.ipiv[gcol] = (int32_t)(p + 1);
          if (zero && *a.info == 0) *a.info = (int32_t)(gcol + 1);
        }
      }
      __syncthreads();
      if (!zero) {
        for (int r = tid; r < nrows; r += PT)
          if (row0 + r > gcol) tile[(size_t)r * jb + c] = pz_mul(tile[(size_t)r * jb + c], s_r);
      }
      __syncthreads();
      // rank-1 update of the panel columns right of c: a_ik -= l_i * u_k
      const int ncols = jb - c - 1;
      if (ncols > 0) {
        for (int idx = tid; idx < nrows * ncols; idx += PT) {
          int r = idx / ncols, k = c + 1 + idx % ncols;
          if (row0 + r <= gcol) continue;
          pz *x = &tile[(size_t)r * jb + k];
          *x = pz_sub(*x, pz_mul(tile[(size_t)r * jb + c], prow[k]));
        }
      }
      __syncthreads();
    } else {
      // ---------------- Cholesky --------------------------------------------
      if (tid == 0) {
        pz d;
        d.s = __ldcg(&a.diag[buf].s);
        d.m = __ldcg(&a.diag[buf].m);
        bool bad = pz_is_nar(d) || pz_is_zero(d) || (d.m >> 31);
        s_flag = bad;
        if (bad) {
          if (g == 0) *a.info = (int32_t)(gcol + 1);
        } else {
          pz sq = pz_sqrt(d);
          s_r = pz_div(pz_one(), sq);
          prow[0] = sq;
        }
      }
      __syncthreads();
      if (s_flag) break;  // leave a_jj = d; the tile is written back below
      if (g == owner_c && tid == 0) tile[(size_t)lrow_c * jb + c] = prow[0];
      for (int r = tid; r < nrows; r += PT)
        if (row0 + r > gcol) tile[(size_t)r * jb + c] = pz_mul(tile[(size_t)r * jb + c], s_r);
      __syncthreads();
      // broadcast l_{k,c} for the panel rows k in (c, jb) held here
      {
        pz *dst = a.xrow + (size_t)buf * jb;
        for (int r = tid; r < nrows; r += PT) {
          int64_t kk = row0 + r - a.j;
          if (kk > c && kk < jb) dst[kk] = tile[(size_t)r * jb + c];
        }
      }
      // the next diagonal element gets its update from column c now, so it
      // can be published at the same barrier
      if (c + 1 < jb) {
        const int owner_n = (int)((c + 1) / R), lrow_n = (c + 1) - owner_n * R;
        if (g == owner_n && tid == 0) {
          pz l = tile[(size_t)lrow_n * jb + c];
          pz *x = &tile[(size_t)lrow_n * jb + c + 1];
          *x = pz_sub(*x, pz_mul(l, l));
          a.diag[buf ^ 1] = *x;
        }
      }
      if (!grid_barrier(a.bar, G, a.err, a.info, kWaitNs)) return;
      const int ncols = jb - c - 1;
      if (ncols > 0) {
        const pz *src = a.xrow + (size_t)buf * jb;
        for (int k = c + 1 + tid; k < jb; k += PT) {
          pz v;
          v.s = __ldcg(&src[k].s);
          v.m = __ldcg(&src[k].m);
          prow[k] = v;
        }
        __syncthreads();
        for (int idx = tid; idx < nrows * ncols; idx += PT) {
          int r = idx / ncols, k = c + 1 + idx % ncols;
          int64_t gr = row0 + r;
          if (gr <= gcol || a.j + k > gr) continue;           // lower triangle only
          if (gr == a.j + c + 1 && k == c + 1) continue;      // done before the barrier
          pz *x = &tile[(size_t)r * jb + k];
          *x = pz_sub(*x, pz_mul(tile[(size_t)r * jb + c], prow[k]));
        }
      }
      __syncthreads();
    }
  }

  // write the panel back
  for (int idx = tid; idx < R * jb; idx += PT) {
    int r, c;
    if (a.trans) { c = idx % jb; r = idx / jb; } else { r = idx % R; c = idx / R; }
    if (r >= nrows) continue;
    int64_t gr = row0 + r, gc = a.j + c;
    if (a.chol && gc > gr) continue;  // never touch the other triangle
    a.A[panel_addr(a, gr, gc)] = pz_to_bits(tile[(size_t)r * jb + c]);
  }
}

// One grid barrier that cannot complete: it waits for one CTA more than the
// grid has, so every CTA's bounded wait runs out after wait_ns, sets the
// error flag and writes POSIT_ERR_TIMEOUT into info (failure detection is
// exercised without a fault or a hang).
__global__ void barrier_timeout_kernel(unsigned *bar, int *err, int32_t *info,
                                       unsigned long long wait_ns) {
  grid_barrier(bar, gridDim.x + 1u, err, info, wait_ns);
}

// The panel's row swaps (pivots k0 .. k1-1) applied to columns [c0, c1).
// LAPACK row swaps k = k0 .. k1-1 (rows k and ipiv[k]-1, in that order) on
// columns [c0, c1).  Each CTA first turns the sequence into one permutation
// of at most 2 (k1 - k0) rows in shared memory: slot t < nk holds row k0 + t,
// and each pivot row outside [k0, k1) gets the slot nk + (first swap that
// names it); the swaps are then played on slot contents.  A warp then moves
// one column at a time: it reads every displaced word, then writes them, so
// a column costs two dependent memory round trips instead of one per swap.
constexpr int LASWP_T = 256;
constexpr int LASWP_MAXK = 256;  // swaps per launch (the panel width kNB)

__global__ void __launch_bounds__(LASWP_T)
laswp_kernel(uint32_t *__restrict__ A, int64_t lda, int64_t c0, int64_t c1, int64_t k0,
             int64_t k1, const int32_t *__restrict__ ipiv) {
  __shared__ int64_t piv[LASWP_MAXK];
  __shared__ int64_t row_of[2 * LASWP_MAXK];   // slot -> matrix row
  __shared__ int32_t slot_of[LASWP_MAXK];      // swap t -> slot of its pivot row
  __shared__ int32_t content[2 * LASWP_MAXK];  // slot -> slot whose old word lands here
  __shared__ int32_t moved[2 * LASWP_MAXK];    // the slots whose word changes
  __shared__ int32_t nmoved;
  __shared__ uint32_t buf[LASWP_T / 32][2 * LASWP_MAXK];
  const int nk = (int)(k1 - k0);
  const int tid = threadIdx.x;
  for (int t = tid; t < nk; t += LASWP_T) piv[t] = (int64_t)ipiv[k0 + t] - 1;
  __syncthreads();
  for (int t = tid; t < nk; t += LASWP_T) {
    const int64_t p = piv[t];
    int slot;
    if (p >= k0 && p < k1) {
      slot = (int)(p - k0);
    } else {
      int first = t;
      for (int u = 0; u < t; ++u)
        if (piv[u] == p) { first = u; break; }
      slot = nk + first;
    }
    slot_of[t] = slot;
    row_of[t] = k0 + t;
    row_of[nk + t] = p;
    content[t] = t;
    content[nk + t] = nk + t;
  }
  __syncthreads();
  if (tid == 0) {
    for (int t = 0; t < nk; ++t) {
      const int o = slot_of[t];
      const int c = content[t];
      content[t] = content[o];
      content[o] = c;
    }
    int cnt = 0;
    for (int sl = 0; sl < 2 * nk; ++sl)
      if (content[sl] != sl) moved[cnt++] = sl;
    nmoved = cnt;
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  const int nm = nmoved;
  uint32_t *wb = buf[warp];
  const int64_t nwarps = (int64_t)gridDim.x * (LASWP_T / 32);
  for (int64_t col = c0 + (int64_t)blockIdx.x * (LASWP_T / 32) + warp; col < c1; col += nwarps) {
    uint32_t *cp = A + col * lda;
    for (int i = lane; i < nm; i += 32) wb[i] = cp[row_of[content[moved[i]]]];
    __syncwarp();
    for (int i = lane; i < nm; i += 32) cp[row_of[moved[i]]] = wb[i];
    __syncwarp();
  }
}

// U12 <- L11^-1 A12 with L11 unit lower (jb x jb at (j, j), jb <= 256), A12 =
// rows [j, j+jb) of columns [c0, c1).  Element (r, col) of U12 receives
// l_{r,t} * u_{t,col} for t = 0 .. r-1 in ascending order.
//
// One warp per column: lane l keeps rows l, l+32, ... of its column in
// registers, u_t is broadcast by a shuffle from the lane that owns row t, so
// the warps never wait for each other; a CTA of 8 warps shares 16 columns of
// L11 at a time, decoded in shared memory.
constexpr int TRSM_T = 256;
constexpr int TRSM_CHUNK = 16;
constexpr int TRSM_MAXJB = 256;

// A value that is not zero and has its scale outside [-lim, lim] (NaR too).
__device__ __forceinline__ bool trsm_outside(pz v, int lim) {
  return !pz_is_zero(v) && (v.s < -lim || v.s > lim);
}

__global__ void __launch_bounds__(TRSM_T)
trsm_llu_kernel(uint32_t *__restrict__ A, int64_t lda, int64_t j, int jb, int64_t c0, int64_t c1,
                uint32_t neg1) {
  // neg1 = 0xFFFFFFFF: the multiplier of the in-band addition's operand pick
  // (pz_add_inband_blend), an argument so that it stays a multiply-add
  __shared__ pz Ls[TRSM_CHUNK][TRSM_MAXJB];  // Ls[u][r] = l_{r, t0+u}
  __shared__ pz_rtab tab_in[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t col = c0 + (int64_t)blockIdx.x * (TRSM_T / 32) + warp;
  const bool active = col < c1;  // warp-uniform
  for (int i = tid; i < 256; i += TRSM_T) tab_in[i] = pz_rtab_inband_entry(i);
  uint32_t *cp = A + j + col * lda;
  pz xs[TRSM_MAXJB / 32];
  bool far = false;
#pragma unroll
  for (int i = 0; i < TRSM_MAXJB / 32; ++i) {
    const int r = 32 * i + lane;
    xs[i] = (active && r < jb) ? pz_decode(cp[r]) : pz_zero();
    far |= trsm_outside(xs[i], 80);
  }
  // In-band steps (the bound argument of the Rgemm kernel): while every
  // product has operands l_{r,t}, u_t that are zero or of scale in [-40, 40]
  // and the column's values started at scales within [-80, 80], every value
  // of the column stays a multiple of 2^-107 below 2^89, so no rounding needs
  // the test for the regimes of 28 or more bits.  So the checks are: the
  // column once (and again after any general step), the chunk of L11 when it
  // is loaded, and u_t -- a column value used as a multiplier -- at its step.
  bool chain_ok = !__any_sync(0xFFFFFFFFu, far);
#pragma unroll
  for (int i0 = 0; i0 < TRSM_MAXJB / 32; ++i0) {
    if (32 * i0 >= jb - 1) break;  // rows from 32*i0 on have nothing below them to update
#pragma unroll 1
    for (int h = 0; h < 32 / TRSM_CHUNK; ++h) {
      const int t0 = 32 * i0 + TRSM_CHUNK * h;
      if (t0 >= jb - 1) break;
      __syncthreads();
      bool l_bad = false;
      for (int idx = tid; idx < TRSM_CHUNK * jb; idx += TRSM_T) {
        const int u = idx / jb, r = idx - u * jb;
        const int t = t0 + u;
        const pz v = (r > t && t < jb) ? pz_decode(A[(j + r) + (j + t) * lda]) : pz_zero();
        l_bad |= trsm_outside(v, 40);
        Ls[u][r] = v;
      }
      const bool l_ok = !__syncthreads_or(l_bad);
      if (active) {
        const int un = min(TRSM_CHUNK, jb - 1 - t0);
        for (int u = 0; u < un; ++u) {
          const int t = t0 + u;
          const int owner = t & 31;
          const pz xt{__shfl_sync(0xFFFFFFFFu, xs[i0].s, owner),
                      __shfl_sync(0xFFFFFFFFu, xs[i0].m, owner)};
          if (l_ok && chain_ok && !trsm_outside(xt, 40)) {  // warp-uniform
#pragma unroll
            for (int i = i0; i < TRSM_MAXJB / 32; ++i) {
              const int r = 32 * i + lane;
              if (r > t && r < jb) {
                const pz p = pz_mul_inband(tab_in, Ls[u][r], xt);
                xs[i] = pz_add_inband_blend(tab_in, neg1, xs[i], pz{p.s, p.m ^ 0x80000000u});
              }
            }
          } else {
            far = false;
#pragma unroll
            for (int i = i0; i < TRSM_MAXJB / 32; ++i) {
              const int r = 32 * i + lane;
              if (r > t && r < jb) xs[i] = pz_sub(xs[i], pz_mul(Ls[u][r], xt));
              far |= trsm_outside(xs[i], 80);
            }
            chain_ok = !__any_sync(0xFFFFFFFFu, far);  // a new start for the argument
          }
        }
      }
    }
  }
  if (active) {
#pragma unroll
    for (int i = 0; i < TRSM_MAXJB / 32; ++i) {
      const int r = 32 * i + lane;
      if (r < jb) cp[r] = pz_to_bits(xs[i]);
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct Scratch {
  void *base = nullptr;
  unsigned *bar;
  int *err;
  uint64_t *cand_key;
  int64_t *cand_row;
  pz *cand_vals;
  pz *xrow;
  pz *diag;
  size_t bytes = 0;
};

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

size_t scratch_bytes(int Gmax, int jbmax) {
  return align_up(4 * sizeof(unsigned)) + align_up(2 * (size_t)Gmax * 8) +
         align_up(2 * (size_t)Gmax * 8) + align_up(2 * (size_t)Gmax * jbmax * sizeof(pz)) +
         align_up(2 * (size_t)jbmax * sizeof(pz)) + align_up(2 * sizeof(pz));
}

// Carve the scratch pointers out of one block of `bytes` (see scratch_bytes).
void carve(Scratch &s, void *base, int Gmax, int jbmax) {
  char *p = static_cast<char *>(base);
  s.base = base;
  s.bar = reinterpret_cast<unsigned *>(p);
  s.err = reinterpret_cast<int *>(p + 2 * sizeof(unsigned));
  p += align_up(4 * sizeof(unsigned));
  s.cand_key = reinterpret_cast<uint64_t *>(p);
  p += align_up(2 * (size_t)Gmax * 8);
  s.cand_row = reinterpret_cast<int64_t *>(p);
  p += align_up(2 * (size_t)Gmax * 8);
  s.cand_vals = reinterpret_cast<pz *>(p);
  p += align_up(2 * (size_t)Gmax * jbmax * sizeof(pz));
  s.xrow = reinterpret_cast<pz *>(p);
  p += align_up(2 * (size_t)jbmax * sizeof(pz));
  s.diag = reinterpret_cast<pz *>(p);
}

struct DeviceLimits {
  int sms = 0;
  int smem_optin = 0;
};

int device_limits(DeviceLimits &d) {
  int dev;
  if (cudaGetDevice(&dev) != cudaSuccess) return POSIT_ERR_DEVICE;
  if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return POSIT_ERR_DEVICE;
  if (cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
      cudaSuccess)
    return POSIT_ERR_DEVICE;
  return POSIT_OK;
}

constexpr int kNB = 256;        // panel width of the timed path
constexpr int kSub = 32;        // width of the sub-panels factored by the cooperative kernel
constexpr int kMinRows = 32;    // fewest panel rows per CTA worth a CTA

// Shape of one panel launch: G CTAs of R rows, width jb.
struct PanelShape {
  int G, R, jb;
  size_t smem;
};

PanelShape panel_shape(const DeviceLimits &d, int64_t rows, int jb_want, int gmax) {
  PanelShape s;
  int64_t G = min64(min64(d.sms, max64(1, gmax)), max64(1, ceil_div(rows, kMinRows)));
  int64_t R = ceil_div(rows, G);
  int jb = jb_want;
  // shared memory: R x jb tile + one row, decoded (8 bytes per element)
  size_t cap = (size_t)d.smem_optin - 1024;
  while (jb > 8 && ((size_t)R * jb + jb) * sizeof(pz) > cap) jb -= 8;
  s.G = (int)G;
  s.R = (int)R;
  s.jb = jb;
  s.smem = ((size_t)R * jb + jb) * sizeof(pz);
  return s;
}

int launch_panel(PanelArgs &pa, const PanelShape &ps, cudaStream_t stream) {
  if (cudaFuncSetAttribute(panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ps.smem) != cudaSuccess)
    return POSIT_ERR_CUDA;
  // the grid barrier's arrival counter starts at zero in every launch
  if (cudaMemsetAsync(pa.bar, 0, sizeof(unsigned), stream) != cudaSuccess) return POSIT_ERR_CUDA;
  pa.jb = ps.jb;
  pa.R = ps.R;
  void *args[] = {&pa};
  cudaError_t e = cudaLaunchCooperativeKernel((const void *)panel_kernel, dim3(ps.G), dim3(PT),
                                              args, ps.smem, stream);
  return e == cudaSuccess ? POSIT_OK : POSIT_ERR_CUDA;
}

int trsm_llu(uint32_t *A, int64_t lda, int64_t j, int jb, int64_t c0, int64_t c1,
             cudaStream_t stream) {
  if (c1 <= c0 || jb <= 1) return POSIT_OK;
  if (jb > TRSM_MAXJB) return POSIT_ERR_DEVICE;  // never: panels are at most kNB wide
  dim3 grid((unsigned)ceil_div(c1 - c0, TRSM_T / 32));
  trsm_llu_kernel<<<grid, TRSM_T, 0, stream>>>(A, lda, j, jb, c0, c1, 0xFFFFFFFFu);
  return launch_status();
}

int laswp(uint32_t *A, int64_t lda, int64_t c0, int64_t c1, int64_t k0, int64_t k1,
          const int32_t *ipiv, cudaStream_t stream) {
  if (c1 <= c0 || k1 <= k0) return POSIT_OK;
  if (k1 - k0 > LASWP_MAXK) return POSIT_ERR_DEVICE;  // never: swaps come per panel
  int64_t blocks = min64(ceil_div(c1 - c0, LASWP_T / 32), 152 * 4);
  laswp_kernel<<<(unsigned)blocks, LASWP_T, 0, stream>>>(A, lda, c0, c1, k0, k1, ipiv);
  return launch_status();
}

}  // namespace

// Lookahead.  With a side stream, the factorisation runs two streams: after
// panel j is applied (its swaps, U12 and the trailing update), the update of
// the NEXT panel's columns is issued first, then that panel is factored on
// the side stream while the caller's stream updates the rest of the trailing
// matrix; the two meet (events) before the next panel's swaps.  The panel
// and the rest touch disjoint columns, and every element still receives its
// updates in ascending column order, so the bits are those of the one-stream
// schedule.  The side stream has the highest priority, so the panel's CTAs
// are scheduled ahead of the trailing Rgemm's as SMs free up.
namespace {

struct Join {
  cudaEvent_t ev[2] = {nullptr, nullptr};
  ~Join() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
  int init() {
    for (cudaEvent_t &e : ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return POSIT_ERR_CUDA;
    return POSIT_OK;
  }
  // `to` waits for the work issued so far on `from` (event slot k)
  int fork(cudaStream_t from, cudaStream_t to, int k) {
    if (cudaEventRecord(ev[k], from) != cudaSuccess) return POSIT_ERR_CUDA;
    return cudaStreamWaitEvent(to, ev[k], 0) == cudaSuccess ? POSIT_OK : POSIT_ERR_CUDA;
  }
};

// CTAs of a panel factored on the side stream: fewer than the SMs, so that
// the trailing Rgemm keeps most of the GPU (measured at n = 8192: Rgetrf
// 442 / 440 / 457 ms with 76 / 38 / 19 CTAs against 445 ms with 152;
// Rpotrf 227 / 227 / 244 ms against 229 ms).
constexpr int kSidePanelCtasLU = 38;
constexpr int kSidePanelCtasChol = 76;

}  // namespace

// LU of the panel's columns [j, j + jb) (rows j .. m-1): sub-panels of kSub
// columns by the cooperative kernel, the rest of the panel brought up to
// date after each by its row swaps, a small unit-lower trsm and a rank-kSub
// Rgemm.  Touches only the panel's columns, ipiv[j .. j+jb) and info.
static int getrf_panel(const DeviceLimits &d, const Scratch &s, int64_t m, int64_t j, int64_t jb,
                       uint32_t *A, int64_t lda, int32_t *ipiv, int32_t *info, int gmax,
                       cudaStream_t stream) {
  int st;
  for (int64_t sp = j; sp < j + jb;) {
    PanelShape ps = panel_shape(d, m - sp, (int)min64(kSub, j + jb - sp), gmax);
    const int w = ps.jb;
    PanelArgs pa{};
    pa.A = A; pa.lda = lda; pa.m = m; pa.j = sp; pa.trans = 0; pa.chol = 0;
    pa.ipiv = ipiv; pa.info = info;
    pa.bar = s.bar; pa.err = s.err; pa.cand_key = s.cand_key; pa.cand_row = s.cand_row;
    pa.cand_vals = s.cand_vals; pa.xrow = s.xrow; pa.diag = s.diag;
    if ((st = launch_panel(pa, ps, stream))) return st;
    // the sub-panel's swaps on the rest of the panel
    if ((st = laswp(A, lda, j, sp, sp, sp + w, ipiv, stream))) return st;
    if ((st = laswp(A, lda, sp + w, j + jb, sp, sp + w, ipiv, stream))) return st;
    if (sp + w < j + jb) {
      if ((st = trsm_llu(A, lda, sp, w, sp + w, j + jb, stream))) return st;
      if (sp + w < m) {
        st = rgemm_launch(false, false, TRI_FULL, m - sp - w, j + jb - sp - w, w, 0xC0000000u,
                          A + (sp + w) + sp * lda, lda, A + sp + (sp + w) * lda, lda,
                          PZ_ONE_BITS, A + (sp + w) + (sp + w) * lda, lda, stream);
        if (st) return st;
      }
    }
    sp += w;
  }
  return POSIT_OK;
}

// Blocked LU on a caller-provided scratch block (bytes from getrf_scratch_bytes).
// Two levels: panels of up to kNB columns drive the big trailing Rgemm; each
// panel is factored by getrf_panel.  Every element still receives its
// updates one column at a time in ascending order, so the factors are those
// of the unblocked algorithm.  side != nullptr: lookahead on that stream.
int getrf_run(int64_t m, int64_t n, uint32_t *A, int64_t lda, int32_t *ipiv, int32_t *info,
              void *scratch, cudaStream_t stream, cudaStream_t side) {
  DeviceLimits d;
  int st = device_limits(d);
  if (st) return st;
  const int64_t mn = min64(m, n);
  Scratch s;
  carve(s, scratch, d.sms, kNB);
  if (cudaMemsetAsync(scratch, 0, scratch_bytes(d.sms, kNB), stream) != cudaSuccess)
    return POSIT_ERR_CUDA;
  const int gmax_side = kSidePanelCtasLU;
  Join join;
  if (side && (st = join.init())) return st;
  bool on_side = false;  // panel j was factored on the side stream
  for (int64_t j = 0; j < mn;) {
    const int64_t jb = min64(kNB, mn - j);
    if (on_side) {
      if ((st = join.fork(side, stream, 1))) return st;
    } else if ((st = getrf_panel(d, s, m, j, jb, A, lda, ipiv, info, d.sms, stream))) {
      return st;
    }
    on_side = false;
    // the panel's swaps on the columns left and right of it
    if ((st = laswp(A, lda, 0, j, j, j + jb, ipiv, stream))) return st;
    if ((st = laswp(A, lda, j + jb, n, j, j + jb, ipiv, stream))) return st;
    if (j + jb < n) {
      if ((st = trsm_llu(A, lda, j, (int)jb, j + jb, n, stream))) return st;
      if (j + jb < m) {
        // next panel's columns first when it is factored ahead
        const int64_t j2 = j + jb, jb2 = min64(kNB, mn - j2);
        const bool ahead = side && jb2 > 0 && j2 + jb2 < n;
        const int64_t c1 = ahead ? j2 + jb2 : n;
        st = rgemm_launch(false, false, TRI_FULL, m - j2, c1 - j2, jb, 0xC0000000u,
                          A + j2 + j * lda, lda, A + j + j2 * lda, lda,
                          PZ_ONE_BITS, A + j2 + j2 * lda, lda, stream);
        if (st) return st;
        if (ahead) {
          if ((st = join.fork(stream, side, 0))) return st;
          if ((st = getrf_panel(d, s, m, j2, jb2, A, lda, ipiv, info, gmax_side, side)))
            return st;
          on_side = true;
          st = rgemm_launch(false, false, TRI_FULL, m - j2, n - c1, jb, 0xC0000000u,
                            A + j2 + j * lda, lda, A + j + c1 * lda, lda,
                            PZ_ONE_BITS, A + j2 + c1 * lda, lda, stream);
          if (st) return st;
        }
      }
    }
    j += jb;
  }
  if (on_side && (st = join.fork(side, stream, 1))) return st;
  return POSIT_OK;
}

size_t getrf_scratch_bytes() {
  DeviceLimits d;
  if (device_limits(d)) return 0;
  return scratch_bytes(d.sms, kNB);
}

// Cholesky of the panel's columns [j, j + jb): sub-panels of kSub columns by
// the cooperative kernel, the rest of the panel updated by Rgemm restricted
// to the factor's triangle.  Touches only the panel's columns (rows for
// upper storage) and info.
static int potrf_panel(const DeviceLimits &d, const Scratch &s, bool upper, int64_t n, int64_t j,
                       int64_t jb, uint32_t *A, int64_t lda, int32_t *info, int gmax,
                       cudaStream_t stream);

// A(t0.., t0..c1) -= F(t0.., c0..c0+kw) F(t0..c1, c0..c0+kw)^T on the lower
// triangle (or the transposed mirror for upper storage); skipped on the
// device once info is set.
static int chol_tri_update(bool upper, int64_t n, uint32_t *A, int64_t lda, int32_t *info,
                           int64_t t0, int64_t c1, int64_t c0, int64_t kw, cudaStream_t stream) {
  const int64_t rows = n - t0, cols = c1 - t0;
  if (rows <= 0 || cols <= 0) return POSIT_OK;
  if (!upper)
    return rgemm_launch_guarded(false, true, TRI_LOWER, rows, cols, kw, 0xC0000000u,
                                A + t0 + c0 * lda, lda, A + t0 + c0 * lda, lda, PZ_ONE_BITS,
                                A + t0 + t0 * lda, lda, info, stream);
  return rgemm_launch_guarded(true, false, TRI_UPPER, cols, rows, kw, 0xC0000000u,
                              A + c0 + t0 * lda, lda, A + c0 + t0 * lda, lda, PZ_ONE_BITS,
                              A + t0 + t0 * lda, lda, info, stream);
}

static int potrf_panel(const DeviceLimits &d, const Scratch &s, bool upper, int64_t n, int64_t j,
                       int64_t jb, uint32_t *A, int64_t lda, int32_t *info, int gmax,
                       cudaStream_t stream) {
  int st;
  for (int64_t sp = j; sp < j + jb;) {
    PanelShape ps = panel_shape(d, n - sp, (int)min64(kSub, j + jb - sp), gmax);
    const int w = ps.jb;
    PanelArgs pa{};
    pa.A = A; pa.lda = lda; pa.m = n; pa.j = sp; pa.trans = upper ? 1 : 0; pa.chol = 1;
    pa.ipiv = nullptr; pa.info = info;
    pa.bar = s.bar; pa.err = s.err; pa.cand_key = s.cand_key; pa.cand_row = s.cand_row;
    pa.cand_vals = s.cand_vals; pa.xrow = s.xrow; pa.diag = s.diag;
    if ((st = launch_panel(pa, ps, stream))) return st;
    // rest of the panel
    if ((st = chol_tri_update(upper, n, A, lda, info, sp + w, j + jb, sp, w, stream))) return st;
    sp += w;
  }
  return POSIT_OK;
}

// Blocked Cholesky: panels of up to kNB columns by potrf_panel, the trailing
// triangle by Rgemm restricted to the factor's triangle.  side != nullptr:
// lookahead as in getrf_run (the next panel's columns are updated first).
int potrf_run(bool upper, int64_t n, uint32_t *A, int64_t lda, int32_t *info, void *scratch,
              cudaStream_t stream, cudaStream_t side) {
  DeviceLimits d;
  int st = device_limits(d);
  if (st) return st;
  Scratch s;
  carve(s, scratch, d.sms, kNB);
  if (cudaMemsetAsync(scratch, 0, scratch_bytes(d.sms, kNB), stream) != cudaSuccess)
    return POSIT_ERR_CUDA;
  const int gmax_side = kSidePanelCtasChol;
  Join join;
  if (side && (st = join.init())) return st;
  bool on_side = false;
  for (int64_t j = 0; j < n;) {
    const int64_t jb = min64(kNB, n - j);
    if (on_side) {
      if ((st = join.fork(side, stream, 1))) return st;
    } else if ((st = potrf_panel(d, s, upper, n, j, jb, A, lda, info, d.sms, stream))) {
      return st;
    }
    on_side = false;
    const int64_t j2 = j + jb, jb2 = min64(kNB, n - j2);
    const bool ahead = side && jb2 > 0 && j2 + jb2 < n;
    // trailing triangle: the next panel's columns first when it goes ahead
    if ((st = chol_tri_update(upper, n, A, lda, info, j2, ahead ? j2 + jb2 : n, j, jb, stream)))
      return st;
    if (ahead) {
      if ((st = join.fork(stream, side, 0))) return st;
      if ((st = potrf_panel(d, s, upper, n, j2, jb2, A, lda, info, gmax_side, side))) return st;
      on_side = true;
      if ((st = chol_tri_update(upper, n, A, lda, info, j2 + jb2, n, j, jb, stream))) return st;
    }
    j += jb;
  }
  if (on_side && (st = join.fork(side, stream, 1))) return st;
  return POSIT_OK;
}

size_t potrf_scratch_bytes() { return getrf_scratch_bytes(); }

cudaStream_t lookahead_stream() {
  static std::mutex mu;
  static cudaStream_t streams[64];
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!streams[dev]) {
    int least = 0, greatest = 0;
    cudaStream_t s = nullptr;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, greatest) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    streams[dev] = s;
  }
  return streams[dev];
}

}  // namespace posit

using namespace posit;

namespace {
int with_scratch(size_t bytes, cudaStream_t stream, void **out) {
  if (cudaMallocAsync(out, bytes, stream) != cudaSuccess) {
    cudaGetLastError();
    return POSIT_ERR_ALLOC;
  }
  return POSIT_OK;
}
}  // namespace

extern "C" int posit_rgetrf(int64_t m, int64_t n, posit32_t *A, int64_t lda, int32_t *ipiv,
                            int32_t *info, cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (lda < max64(1, m)) return -4;
  if (!info) return -6;
  if (m > 0 && n > 0 && !A) return -3;
  if (m > 0 && n > 0 && !ipiv) return -5;
  if (cudaMemsetAsync(info, 0, sizeof(int32_t), stream) != cudaSuccess) return POSIT_ERR_CUDA;
  if (m == 0 || n == 0) return POSIT_OK;
  size_t bytes = getrf_scratch_bytes();
  if (!bytes) return POSIT_ERR_DEVICE;
  void *scratch = nullptr;
  int st = with_scratch(bytes, stream, &scratch);
  if (st) return st;
  st = getrf_run(m, n, A, lda, ipiv, info, scratch, stream, lookahead_stream());
  cudaFreeAsync(scratch, stream);
  return st;
}

extern "C" int posit_rpotrf(char uplo, int64_t n, posit32_t *A, int64_t lda, int32_t *info,
                            cudaStream_t stream) {
  if (!is_lower(uplo) && !is_upper(uplo)) return -1;
  if (n < 0) return -2;
  if (lda < max64(1, n)) return -4;
  if (!info) return -5;
  if (n > 0 && !A) return -3;
  if (cudaMemsetAsync(info, 0, sizeof(int32_t), stream) != cudaSuccess) return POSIT_ERR_CUDA;
  if (n == 0) return POSIT_OK;
  size_t bytes = potrf_scratch_bytes();
  if (!bytes) return POSIT_ERR_DEVICE;
  void *scratch = nullptr;
  int st = with_scratch(bytes, stream, &scratch);
  if (st) return st;
  st = potrf_run(is_upper(uplo), n, A, lda, info, scratch, stream, lookahead_stream());
  cudaFreeAsync(scratch, stream);
  return st;
}

extern "C" int posit_selftest_wait(int64_t wait_ns, int32_t *info, cudaStream_t stream) {
  if (wait_ns < 1000 || wait_ns > 10000000000ll) return -1;
  if (!info) return -2;
  if (cudaMemsetAsync(info, 0, sizeof(int32_t), stream) != cudaSuccess) return POSIT_ERR_CUDA;
  void *scratch = nullptr;
  int st = with_scratch(256, stream, &scratch);
  if (st) return st;
  unsigned *bar = static_cast<unsigned *>(scratch);
  int *err = reinterpret_cast<int *>(bar + 2);
  st = POSIT_OK;
  if (cudaMemsetAsync(scratch, 0, 256, stream) != cudaSuccess) {
    st = POSIT_ERR_CUDA;
  } else {
    barrier_timeout_kernel<<<2, PT, 0, stream>>>(bar, err, info, (unsigned long long)wait_ns);
    st = launch_status();
  }
  cudaFreeAsync(scratch, stream);
  return st;
}
