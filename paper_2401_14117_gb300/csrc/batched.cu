// batched.cu -- many independent Rgetrf+Rgetrs / Rpotrf+Rpotrs problems in
// one persistent launch.
//
// A persistent grid of CTAs pulls problem indices from an atomic counter, in
// the order given by the plan (largest n first, so the longest problems start
// first).  Each CTA factors and solves one problem at a time, with the matrix
// decoded (scale, significand pairs) either in shared memory, when n*n*8
// bytes fit the plan's shared-memory budget, or in the CTA's slice of a
// global workspace.  The per-element operation order is the unblocked order
// of Rgetrf/Rpotrf and the trsm orders of Rgetrs/Rpotrs (see
// include/posit_gb300.h), so every result equals the plain routines' result
// bit for bit, whatever the plan.
#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "chain.cuh"

namespace posit {
namespace {

struct Key {
  uint64_t k;
  int r;
};

__device__ __forceinline__ uint64_t abs_key(pz a) {
  if (pz_is_nar(a)) return ~0ull;
  if (pz_is_zero(a)) return 1ull;
  return ((uint64_t)(uint32_t)(a.s + (1 << 24)) << 32) | (uint64_t)(a.m & 0x7FFFFFFFu);
}

__device__ __forceinline__ bool key_better(uint64_t k1, int r1, uint64_t k2, int r2) {
  return k1 > k2 || (k1 == k2 && r1 < r2);
}

// Block-wide argmax of (key, lowest row); returns the winner in every thread.
__device__ Key block_argmax(uint64_t k, int r, Key *red) {
  for (int off = 16; off > 0; off >>= 1) {
    uint64_t ok = __shfl_down_sync(0xFFFFFFFFu, k, off);
    int orow = __shfl_down_sync(0xFFFFFFFFu, r, off);
    if (key_better(ok, orow, k, r)) { k = ok; r = orow; }
  }
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = Key{k, r};
  __syncthreads();
  if (threadIdx.x == 0) {
    Key b = red[0];
    for (int i = 1; i < nw; ++i)
      if (key_better(red[i].k, red[i].r, b.k, b.r)) b = red[i];
    red[32] = b;
  }
  __syncthreads();
  Key out = red[32];
  __syncthreads();
  return out;
}

// One rounded multiply and one rounded subtract, x - a*b.  FAST uses the
// per-scale rounding table and is exact for operands that are not NaR (a
// problem whose matrix holds no NaR never creates one while it is factored:
// zero pivots are skipped and Cholesky stops at the first d <= 0); otherwise
// the general operations propagate NaR.
template <bool FAST>
__device__ __forceinline__ pz sub_mul(const pz_rtab *tab, pz x, pz a, pz b) {
  if (FAST) {
    const pz p = pz_mul_tab(tab, a, b);
    return pz_add_tab(tab, x, pz{p.s, p.m ^ 0x80000000u});
  }
  return pz_sub(x, pz_mul(a, b));
}

template <bool FAST>
__device__ __forceinline__ pz mul_any(const pz_rtab *tab, pz a, pz b) {
  return FAST ? pz_mul_tab(tab, a, b) : pz_mul(a, b);
}

// In-band steps (tables of pz_rtab_inband_entry): one rounded operation whose
// operands are zero or have scales in [-40, 40] (the reciprocal of such a
// pivot: [-41, 40]) never leaves the scales [-107, 82], so it needs no test
// for the regimes of 28 or more bits.  Each column checks that every value
// it is about to use is in band: the trailing entries (checked when the
// previous column updated them) and the scaled column (checked here).
__device__ __forceinline__ bool out_of_band(pz v) {
  return !pz_is_zero(v) && (v.s < -40 || v.s > 40);
}

__device__ __forceinline__ pz sub_mul_inband(const pz_rtab *tab, pz x, pz a, pz b) {
  const pz p = pz_mul_inband(tab, a, b);
  return pz_add_inband(tab, x, pz{p.s, p.m ^ 0x80000000u});
}

// ---------------------------------------------------------------------------
// Blocked factorisations inside one CTA.  Panels of BW columns are factored
// column by column; the rest of the matrix is then brought up to date by a
// register-tiled update in which every element receives the panel's BW terms
// in ascending order, exactly as the unblocked algorithm orders them, so the
// result is the same for every panel width.
// ---------------------------------------------------------------------------
constexpr int BW = 16;             // panel width
constexpr int TTM = 4, TTN = 2;    // register tile of the trailing update

// M(r, c) -= sum_{t < kw} l(r, t) u(t, c), t ascending, for rows [r0, r1) and
// columns [c0, c1) (tri 1: only c <= r; tri 2: only r <= c), with
// l(r, t) = L[(r - r0) * li + t * lt] and u(t, c) = U[t * su + (c - c0) * sk].
// ib: the operands and the starting values are zero or have scales in
// [-40, 40]; then, as in Rgemm, no rounding of the chain can reach the
// regimes of 28 or more bits.  Returns (after a barrier) whether any updated
// value is outside [-40, 40].
template <bool FAST>
__device__ bool trailing_update(pz *M, int n, int r0, int r1, int c0, int c1, const pz *L, int li,
                                int lt, const pz *U, int su, int sk, int kw, int tri,
                                const pz_rtab *tab, const pz_rtab *tab_in, bool ib) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nr = r1 - r0, nc = c1 - c0;
  bool oob = false;
  if (nr > 0 && nc > 0 && kw > 0) {
    const int rs = (nr + TTM - 1) / TTM;  // row stride of a tile: its rows are r0+tr+i*rs
    const int ncol_t = (nc + TTN - 1) / TTN;
    const int tiles = rs * ncol_t;
    for (int tile = tid; tile < tiles; tile += nt) {
      const int tr = tile % rs, tc = tile / rs;
      int rr[TTM], cc[TTN];
      bool ok[TTM][TTN];
      pz acc[TTM][TTN];
#pragma unroll
      for (int i = 0; i < TTM; ++i) rr[i] = tr + i * rs;
#pragma unroll
      for (int j = 0; j < TTN; ++j) cc[j] = tc * TTN + j;
      bool any = false;
#pragma unroll
      for (int i = 0; i < TTM; ++i)
#pragma unroll
        for (int j = 0; j < TTN; ++j) {
          const int r = r0 + rr[i], c = c0 + cc[j];
          ok[i][j] = rr[i] < nr && cc[j] < nc &&
                     (tri == 0 || (tri == 1 ? c <= r : r <= c));
          acc[i][j] = ok[i][j] ? M[r + (size_t)c * n] : pz_one();
          any |= ok[i][j];
        }
      if (!any) continue;
      for (int t = 0; t < kw; ++t) {
        pz l[TTM], u[TTN];
#pragma unroll
        for (int i = 0; i < TTM; ++i)
          l[i] = rr[i] < nr ? L[(size_t)rr[i] * li + (size_t)t * lt] : pz_one();
#pragma unroll
        for (int j = 0; j < TTN; ++j)
          u[j] = cc[j] < nc ? U[(size_t)t * su + (size_t)cc[j] * sk] : pz_one();
        if (FAST && ib) {
#pragma unroll
          for (int i = 0; i < TTM; ++i)
#pragma unroll
            for (int j = 0; j < TTN; ++j) acc[i][j] = sub_mul_inband(tab_in, acc[i][j], l[i], u[j]);
        } else {
#pragma unroll
          for (int i = 0; i < TTM; ++i)
#pragma unroll
            for (int j = 0; j < TTN; ++j) acc[i][j] = sub_mul<FAST>(tab, acc[i][j], l[i], u[j]);
        }
      }
#pragma unroll
      for (int i = 0; i < TTM; ++i)
#pragma unroll
        for (int j = 0; j < TTN; ++j)
          if (ok[i][j]) {
            M[(r0 + rr[i]) + (size_t)(c0 + cc[j]) * n] = acc[i][j];
            oob |= out_of_band(acc[i][j]);
          }
    }
  }
  return __syncthreads_or(oob);
}

// Whether any element of the r x c block at P (element (i, j) at
// P[i * si + j * sj]) is outside [-40, 40], after a barrier.
__device__ bool block_out_of_band(const pz *P, int r, int c, int si, int sj) {
  bool oob = false;
  for (int idx = threadIdx.x; idx < r * c; idx += blockDim.x) {
    const int i = idx % r, j = idx / r;
    oob |= out_of_band(P[(size_t)i * si + (size_t)j * sj]);
  }
  return __syncthreads_or(oob);
}

// LU with partial pivoting of the decoded n x n matrix M (column-major, ld n),
// blocked by BW columns.  ib: every entry starts in band.
template <bool FAST>
__device__ int lu_decoded(pz *M, int n, int32_t *ipiv, Key *red, pz *sh, const pz_rtab *tab,
                          const pz_rtab *tab_in, bool ib) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  int info = 0;
  bool oob = false;
  for (int p0 = 0; p0 < n; p0 += BW) {
    const int pe = min(n, p0 + BW);  // panel columns [p0, pe)
    // ---- the panel, column by column (in-panel updates only)
    for (int c = p0; c < pe; ++c) {
      uint64_t best = 0;
      int brow = 0x7FFFFFFF;
      for (int i = c + tid; i < n; i += nt) {
        uint64_t k = abs_key(M[i + (size_t)c * n]);
        if (key_better(k, i, best, brow)) { best = k; brow = i; }
      }
      Key w = block_argmax(best, brow, red);
      const int p = w.r;
      const bool zero = pz_is_zero(M[p + (size_t)c * n]);
      if (tid == 0) ipiv[c] = p + 1;
      if (zero) {
        if (info == 0) info = c + 1;
      } else {
        if (p != c)  // the whole rows, so the trailing columns are permuted too
          for (int k = tid; k < n; k += nt) {
            pz t = M[c + (size_t)k * n];
            M[c + (size_t)k * n] = M[p + (size_t)k * n];
            M[p + (size_t)k * n] = t;
          }
        __syncthreads();
        // after the swap the pivot sits at (c, c)
        if (tid == 0) sh[0] = pz_div(pz_one(), M[c + (size_t)c * n]);
        __syncthreads();
        const pz r = sh[0];
        for (int i = c + 1 + tid; i < n; i += nt) {
          pz *x = &M[i + (size_t)c * n];
          *x = (FAST && ib) ? pz_mul_inband(tab_in, *x, r) : mul_any<FAST>(tab, *x, r);
          oob |= out_of_band(*x);
        }
      }
      const bool any_oob = __syncthreads_or(oob);  // every thread reaches the barrier
      const bool ib_update = FAST && ib && !any_oob;
      oob = false;
      const pz *lc = M + (size_t)c * n;
      for (int k = c + 1 + warp; k < pe; k += nw) {
        pz *col = M + (size_t)k * n;
        const pz u = col[c];
        if (ib_update) {
          for (int i = c + 1 + lane; i < n; i += 32) {
            col[i] = sub_mul_inband(tab_in, col[i], lc[i], u);
            oob |= out_of_band(col[i]);
          }
        } else {
          for (int i = c + 1 + lane; i < n; i += 32) {
            col[i] = sub_mul<FAST>(tab, col[i], lc[i], u);
            oob |= out_of_band(col[i]);
          }
        }
      }
      // ib keeps describing the trailing entries the later panel columns use
      const bool upd_oob = __syncthreads_or(oob);  // every thread reaches the barrier
      ib = ib && !upd_oob && !any_oob;
      oob = false;
    }
    if (pe >= n) break;
    // ---- U12: rows [p0, pe) of the columns right of the panel; one thread
    // per column, t ascending for every row
    for (int k = pe + tid; k < n; k += nt) {
      pz *col = M + (size_t)k * n;
      for (int r = p0 + 1; r < pe; ++r) {
        pz x = col[r];
        for (int t = p0; t < r; ++t) x = sub_mul<FAST>(tab, x, M[r + (size_t)t * n], col[t]);
        col[r] = x;
      }
    }
    __syncthreads();
    // ---- A22 -= L21 U12 (K = pe - p0)
    const bool l21_oob = block_out_of_band(M + pe + (size_t)p0 * n, n - pe, pe - p0, 1, n);
    const bool u12_oob = block_out_of_band(M + p0 + (size_t)pe * n, pe - p0, n - pe, 1, n);
    const bool ops_in = !l21_oob && !u12_oob;
    const bool a22_oob = trailing_update<FAST>(M, n, pe, n, pe, n, M + pe + (size_t)p0 * n, 1, n,
                                               M + p0 + (size_t)pe * n, 1, n, pe - p0, 0, tab,
                                               tab_in, FAST && ib && ops_in);
    ib = !a22_oob;
  }
  return info;
}

// Cholesky (lower) of the decoded matrix, blocked by BW columns; returns info.
template <bool FAST>
__device__ int chol_decoded(pz *M, int n, pz *sh, const pz_rtab *tab, const pz_rtab *tab_in,
                            bool ib) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  bool oob = false;
  for (int p0 = 0; p0 < n; p0 += BW) {
    const int pe = min(n, p0 + BW);
    for (int j = p0; j < pe; ++j) {
      pz d = M[j + (size_t)j * n];
      if (pz_is_nar(d) || pz_is_zero(d) || (d.m >> 31)) {
        // leave the trailing triangle as the unblocked algorithm does: with
        // the updates of the panel's completed columns p0 .. j-1
        if (pe < n)
          trailing_update<FAST>(M, n, pe, n, pe, n, M + pe + (size_t)p0 * n, 1, n,
                                M + pe + (size_t)p0 * n, n, 1, j - p0, 1, tab, tab_in, false);
        return j + 1;
      }
      if (tid == 0) {
        pz s = pz_sqrt(d);
        sh[0] = s;
        sh[1] = pz_div(pz_one(), s);
      }
      __syncthreads();
      if (tid == 0) M[j + (size_t)j * n] = sh[0];
      const pz r = sh[1];
      for (int i = j + 1 + tid; i < n; i += nt) {
        pz *x = &M[i + (size_t)j * n];
        *x = (FAST && ib) ? pz_mul_inband(tab_in, *x, r) : mul_any<FAST>(tab, *x, r);
        oob |= out_of_band(*x);
      }
      const bool any_oob = __syncthreads_or(oob);  // every thread reaches the barrier
      const bool ib_update = FAST && ib && !any_oob;
      oob = false;
      // a_ik -= l_ij l_kj for the panel columns k in (j, pe), rows i >= k
      const pz *lj = M + (size_t)j * n;
      for (int k = j + 1 + warp; k < pe; k += nw) {
        pz *col = M + (size_t)k * n;
        const pz u = lj[k];
        if (ib_update) {
          for (int i = k + lane; i < n; i += 32) {
            col[i] = sub_mul_inband(tab_in, col[i], lj[i], u);
            oob |= out_of_band(col[i]);
          }
        } else {
          for (int i = k + lane; i < n; i += 32) {
            col[i] = sub_mul<FAST>(tab, col[i], lj[i], u);
            oob |= out_of_band(col[i]);
          }
        }
      }
      const bool upd_oob = __syncthreads_or(oob);  // every thread reaches the barrier
      ib = ib && !upd_oob && !any_oob;
      oob = false;
    }
    if (pe >= n) break;
    // the trailing lower triangle: a_ik -= sum_t l_it l_kt, t ascending
    const pz *L21 = M + pe + (size_t)p0 * n;
    const bool ops_in = !block_out_of_band(L21, n - pe, pe - p0, 1, n);
    const bool a22_oob = trailing_update<FAST>(M, n, pe, n, pe, n, L21, 1, n, L21, n, 1, pe - p0,
                                               1, tab, tab_in, FAST && ib && ops_in);
    ib = !a22_oob;
  }
  return 0;
}

// Rpotrs 'U' on the decoded factor: U^T y = b (updates from k ascending,
// then / u_ii), U x = y (updates from k descending, then / u_ii); both run
// column by column with the rows in parallel.  The factor is held transposed:
// u_ik = M[k + i * n] (the lower triangle of M is U^T).
__device__ void potrs_decoded_upper(const pz *M, int n, pz *X, int nrhs) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = 0; k < n; ++k) {
    for (int c = tid; c < nrhs; c += nt) X[k + c * n] = pz_div(X[k + c * n], M[k + (size_t)k * n]);
    __syncthreads();
    const int m = n - k - 1;
    for (int idx = tid; idx < m * nrhs; idx += nt) {
      int i = k + 1 + idx % m, c = idx / m;
      X[i + c * n] = pz_sub(X[i + c * n], pz_mul(M[i + (size_t)k * n], X[k + c * n]));
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    for (int c = tid; c < nrhs; c += nt) X[k + c * n] = pz_div(X[k + c * n], M[k + (size_t)k * n]);
    __syncthreads();
    for (int idx = tid; idx < k * nrhs; idx += nt) {
      int i = idx % k, c = idx / k;
      X[i + c * n] = pz_sub(X[i + c * n], pz_mul(M[k + (size_t)i * n], X[k + c * n]));
    }
    __syncthreads();
  }
}

// Rgetrs 'N' on decoded factors: swaps, L y = b (unit), U x = y.
__device__ void getrs_decoded(const pz *M, int n, const int32_t *ipiv, pz *X, int nrhs) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int c = tid; c < nrhs; c += nt)
    for (int i = 0; i < n; ++i) {
      int p = ipiv[i] - 1;
      pz t = X[i + c * n];
      X[i + c * n] = X[p + c * n];
      X[p + c * n] = t;
    }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int m = n - j - 1;
    for (int idx = tid; idx < m * nrhs; idx += nt) {
      int i = j + 1 + idx % m, c = idx / m;
      X[i + c * n] = pz_sub(X[i + c * n], pz_mul(M[i + (size_t)j * n], X[j + c * n]));
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    for (int c = tid; c < nrhs; c += nt) X[k + c * n] = pz_div(X[k + c * n], M[k + (size_t)k * n]);
    __syncthreads();
    for (int idx = tid; idx < k * nrhs; idx += nt) {
      int i = idx % k, c = idx / k;
      X[i + c * n] = pz_sub(X[i + c * n], pz_mul(M[i + (size_t)k * n], X[k + c * n]));
    }
    __syncthreads();
  }
}

// Rpotrs 'L' on the decoded factor: L y = b then the dot-form L^T x = y.
__device__ void potrs_decoded(const pz *M, int n, pz *X, int nrhs, pz *prod, const pzs_rtab *tab) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = 0; j < n; ++j) {
    for (int c = tid; c < nrhs; c += nt) X[j + c * n] = pz_div(X[j + c * n], M[j + (size_t)j * n]);
    __syncthreads();
    const int m = n - j - 1;
    for (int idx = tid; idx < m * nrhs; idx += nt) {
      int i = j + 1 + idx % m, c = idx / m;
      X[i + c * n] = pz_sub(X[i + c * n], pz_mul(M[i + (size_t)j * n], X[j + c * n]));
    }
    __syncthreads();
  }
  // x_i = (y_i - sum_{k>i, ascending} l_ki x_k) / l_ii: products in parallel,
  // stored negated in the signed chain form (chain.cuh), one serial chain per
  // right-hand side in checked runs of PZS_RUN links; a row with a product
  // that is NaR or outside the chain band runs on the general addition (a
  // NaR product or y_i makes x_i NaR there)
  pzs *pr_all = reinterpret_cast<pzs *>(prod);
  for (int i = n - 1; i >= 0; --i) {
    const int m = n - i - 1;
    int bad = 0;
    for (int idx = tid; idx < m * nrhs; idx += nt) {
      int k = i + 1 + idx % m, c = idx / m;
      const pz p = pz_mul(M[k + (size_t)i * n], X[k + c * n]);
      const pzs q = pzs_of(pz{p.s, p.m ^ 0x80000000u});
      bad |= !pzs_in_band(q);
      pr_all[idx] = q;
    }
    const bool products_ok = !__syncthreads_or(bad);
    for (int c = tid; c < nrhs; c += nt) {
      pzs acc = pzs_of(X[i + c * n]);
      const pzs *pr = pr_all + c * m;
      int t = 0;
      for (; t + PZS_RUN <= m; t += PZS_RUN) pzs_run<PZS_RUN>(acc, pr + t, PZS_RUN, tab, products_ok);
      if (t < m) pzs_run<0>(acc, pr + t, m - t, tab, products_ok);
      X[i + c * n] = pz_div(pz_of(acc), M[i + (size_t)i * n]);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(512) batched_kernel(const posit_problem *__restrict__ probs,
                               const int32_t *__restrict__ order, int64_t count,
                               unsigned long long *counter, pz *workspace,
                               size_t ws_elems_per_cta, int smem_elems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pz *sm = reinterpret_cast<pz *>(smem_raw);
  __shared__ Key red[33];
  __shared__ pz sh[2];
  __shared__ long long s_idx;
  __shared__ int s_nar;
  __shared__ pz_rtab rtab[256];
  __shared__ pz_rtab rtab_in[256];
  __shared__ pzs_rtab ctab[256];  // the serial chain's rounding constants
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < 256; i += nt) {
    rtab[i] = pz_rtab_entry(i);
    rtab_in[i] = pz_rtab_inband_entry(i);
    ctab[i] = pzs_rtab_entry(i);
  }
  pz *ws = workspace + (size_t)blockIdx.x * ws_elems_per_cta;
  for (;;) {
    if (tid == 0) {
      unsigned long long i = atomicAdd(counter, 1ull);
      s_idx = (long long)i < count ? (long long)i : -1;
    }
    __syncthreads();
    const long long qi = s_idx;
    __syncthreads();
    if (qi < 0) break;
    const posit_problem P = probs[order ? order[qi] : qi];
    const int n = P.n, nrhs = P.nrhs;
    // M (n x n), X (n x nrhs), then scratch of n * max(nrhs, 1) (the products
    // of the dot-form solve)
    const size_t need = (size_t)n * n + (size_t)n * nrhs + (size_t)n * (nrhs > 1 ? nrhs : 1);
    pz *M = need <= (size_t)smem_elems ? sm : ws;
    pz *X = M + (size_t)n * n;
    pz *prod = X + (size_t)n * nrhs;
    const bool lower_only = P.kind == POSIT_CHOLESKY, upper_only = P.kind == POSIT_CHOLESKY_U;
    if (tid == 0) s_nar = 0;
    __syncthreads();
    int nar = 0, oob = 0;
    // the upper Cholesky is factored as the lower one of the transposed
    // upper triangle (the same operations on mirrored indices): M(i, k) =
    // a(k, i) for i >= k
    for (int idx = tid; idx < n * n; idx += nt) {
      int i = idx % n, k = idx / n;
      bool skip = (lower_only || upper_only) && k > i;
      const uint32_t w =
          skip ? 0u : (upper_only ? P.A[k + (int64_t)i * P.lda] : P.A[i + (int64_t)k * P.lda]);
      nar |= w == PZ_NAR_BITS;
      const pz v = pz_decode(w);
      oob |= out_of_band(v);
      M[idx] = v;
    }
    if (__syncthreads_or(nar) && tid == 0) s_nar = 1;
    const bool ib0 = !__syncthreads_or(oob);
    for (int idx = tid; idx < n * nrhs; idx += nt) {
      int i = idx % n, c = idx / n;
      X[idx] = pz_decode(P.B[i + (int64_t)c * P.ldb]);
    }
    __syncthreads();
    const bool fast = s_nar == 0;  // the matrix holds no NaR
    int info;
    if (P.kind == POSIT_LU) {
      info = fast ? lu_decoded<true>(M, n, P.ipiv, red, sh, rtab, rtab_in, ib0)
                  : lu_decoded<false>(M, n, P.ipiv, red, sh, rtab, rtab_in, false);
      getrs_decoded(M, n, P.ipiv, X, nrhs);
    } else if (P.kind == POSIT_CHOLESKY) {
      info = fast ? chol_decoded<true>(M, n, sh, rtab, rtab_in, ib0)
                  : chol_decoded<false>(M, n, sh, rtab, rtab_in, false);
      if (info == 0) potrs_decoded(M, n, X, nrhs, prod, ctab);
    } else {
      info = fast ? chol_decoded<true>(M, n, sh, rtab, rtab_in, ib0)
                  : chol_decoded<false>(M, n, sh, rtab, rtab_in, false);
      if (info == 0) potrs_decoded_upper(M, n, X, nrhs);
    }
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += nt) {
      int i = idx % n, k = idx / n;
      if ((lower_only || upper_only) && k > i) continue;
      if (upper_only)
        P.A[k + (int64_t)i * P.lda] = pz_to_bits(M[idx]);
      else
        P.A[i + (int64_t)k * P.lda] = pz_to_bits(M[idx]);
    }
    if (P.kind == POSIT_LU || info == 0)
      for (int idx = tid; idx < n * nrhs; idx += nt) {
        int i = idx % n, c = idx / n;
        P.B[i + (int64_t)c * P.ldb] = pz_to_bits(X[idx]);
      }
    if (tid == 0 && P.info) *P.info = info;
    __syncthreads();
  }
}

}  // namespace

size_t batched_ws_elems(int max_n, int max_nrhs) {
  return (size_t)max_n * max_n + (size_t)max_n * max_nrhs +
         (size_t)max_n * (max_nrhs > 1 ? max_nrhs : 1);
}

int batched_launch(const posit_problem *probs, const int32_t *order, int64_t count, int max_n,
                   int max_nrhs, const posit_plan &plan, void *workspace, cudaStream_t stream) {
  int dev, sms;
  if (cudaGetDevice(&dev) != cudaSuccess) return POSIT_ERR_DEVICE;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return POSIT_ERR_DEVICE;
  const int grid = sms * plan.ctas_per_sm;
  unsigned long long *counter = static_cast<unsigned long long *>(workspace);
  pz *ws = reinterpret_cast<pz *>(static_cast<char *>(workspace) + 256);
  const size_t per = batched_ws_elems(max_n, max_nrhs);
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream) != cudaSuccess)
    return POSIT_ERR_CUDA;
  const size_t smem = (size_t)plan.smem_bytes;
  if (cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return POSIT_ERR_CUDA;
  batched_kernel<<<grid, plan.threads, smem, stream>>>(probs, order, count, counter, ws, per,
                                                       (int)(smem / sizeof(pz)));
  return launch_status();
}

size_t batched_workspace_bytes(int max_n, int max_nrhs, const posit_plan &plan) {
  int dev, sms;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return 256 + (size_t)sms * plan.ctas_per_sm * batched_ws_elems(max_n, max_nrhs) * sizeof(pz);
}

}  // namespace posit

using namespace posit;

namespace {
bool plan_ok(const posit_plan *p) {
  return p && p->threads >= 32 && p->threads <= 512 && (p->threads % 32) == 0 &&
         p->ctas_per_sm >= 1 && p->ctas_per_sm <= 32 && p->smem_bytes >= 0 &&
         p->smem_bytes <= 232448;
}
}  // namespace

extern "C" int posit_batched_workspace_size(int64_t max_n, int64_t max_nrhs, const posit_plan *plan,
                                            size_t *bytes) {
  if (max_n < 0) return -1;
  if (max_nrhs < 0) return -2;
  if (!plan_ok(plan)) return -3;
  if (!bytes) return -4;
  *bytes = batched_workspace_bytes((int)max_n, (int)max_nrhs, *plan);
  return *bytes ? POSIT_OK : POSIT_ERR_DEVICE;
}

extern "C" int posit_factor_solve_batched(int64_t count, const posit_problem *problems,
                                          const int32_t *order, int64_t max_n, int64_t max_nrhs,
                                          const posit_plan *plan, void *workspace,
                                          cudaStream_t stream) {
  if (count < 0) return -1;
  if (count > 0 && !problems) return -2;
  if (max_n < 0 || max_n > 46340) return -4;
  if (max_nrhs < 0) return -5;
  if (!plan_ok(plan)) return -6;
  if (count == 0) return POSIT_OK;
  if (!workspace) {
    size_t bytes = batched_workspace_bytes((int)max_n, (int)max_nrhs, *plan);
    void *ws = nullptr;
    if (!bytes) return POSIT_ERR_DEVICE;
    if (cudaMallocAsync(&ws, bytes, stream) != cudaSuccess) {
      cudaGetLastError();
      return POSIT_ERR_ALLOC;
    }
    int st = batched_launch(problems, order, count, (int)max_n, (int)max_nrhs, *plan, ws, stream);
    cudaFreeAsync(ws, stream);
    return st;
  }
  return batched_launch(problems, order, count, (int)max_n, (int)max_nrhs, *plan, workspace, stream);
}

// ---------------------------------------------------------------------------
// Autotuner of the launch shape.  The problems' A and B are packed once into a
// pristine copy; before every timed run the working copy is restored from it
// with one device-to-device copy, so each run factors the same inputs and the
// caller's arrays are never written.
// ---------------------------------------------------------------------------
namespace {

struct TuneArena {
  void *p = nullptr;
  cudaStream_t s = nullptr;
  ~TuneArena() {
    if (p) cudaFreeAsync(p, s);
  }
};

bool plan_less(const posit_plan &a, float ta, const posit_plan &b, float tb) {
  if (ta != tb) return ta < tb;
  const int64_t wa = (int64_t)a.threads * a.ctas_per_sm, wb = (int64_t)b.threads * b.ctas_per_sm;
  if (wa != wb) return wa < wb;
  return a.smem_bytes < b.smem_bytes;
}

}  // namespace

extern "C" int posit_autotune(int64_t count, const posit_problem *problems, const int32_t *order,
                              int64_t max_n, int64_t max_nrhs, const posit_plan *cands,
                              int32_t ncand, int32_t reps, posit_plan *best, float *times_ms,
                              cudaStream_t stream) {
  if (count <= 0) return -1;
  if (!problems) return -2;
  if (max_n < 0 || max_n > 46340) return -4;
  if (max_nrhs < 0) return -5;
  if (!cands || ncand < 1) return -6;
  if (reps < 1) return -8;
  if (!best) return -9;

  // the caller's descriptors, checked before anything is copied
  std::vector<posit_problem> hp((size_t)count);
  if (cudaMemcpyAsync(hp.data(), problems, sizeof(posit_problem) * (size_t)count,
                      cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return POSIT_ERR_CUDA;
  size_t words = 0;  // A and B of every problem, packed with ld = n
  for (const posit_problem &q : hp) {
    if (q.n < 0 || q.n > max_n || q.nrhs < 0 || q.nrhs > max_nrhs || q.lda < (q.n > 0 ? q.n : 1) ||
        q.ldb < (q.n > 0 ? q.n : 1) || !q.A || (q.nrhs > 0 && !q.B) ||
        (q.kind != POSIT_LU && q.kind != POSIT_CHOLESKY && q.kind != POSIT_CHOLESKY_U))
      return -2;
    words += (size_t)q.n * q.n + (size_t)q.n * q.nrhs;
  }
  size_t ipiv_words = 0;
  for (const posit_problem &q : hp) ipiv_words += (size_t)q.n;

  size_t ws_bytes = 0;
  for (int32_t c = 0; c < ncand; ++c)
    if (plan_ok(&cands[c]))
      ws_bytes = std::max(ws_bytes, batched_workspace_bytes((int)max_n, (int)max_nrhs, cands[c]));
  if (ws_bytes == 0) return POSIT_ERR_CUDA;

  // one allocation: pristine A/B | working A/B | ipiv | info | descriptors | workspace
  auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
  const size_t ab_bytes = up16(words * 4);
  const size_t off_work = ab_bytes, off_ipiv = 2 * ab_bytes;
  const size_t off_info = off_ipiv + up16(ipiv_words * 4);
  const size_t off_desc = off_info + up16((size_t)count * 4);
  const size_t off_ws = off_desc + up16(sizeof(posit_problem) * (size_t)count);
  const size_t total = off_ws + ws_bytes;
  TuneArena arena;
  arena.s = stream;
  if (cudaMallocAsync(&arena.p, total, stream) != cudaSuccess) {
    arena.p = nullptr;
    cudaGetLastError();
    return POSIT_ERR_ALLOC;
  }
  char *base = static_cast<char *>(arena.p);
  uint32_t *pristine = reinterpret_cast<uint32_t *>(base);
  uint32_t *work = reinterpret_cast<uint32_t *>(base + off_work);
  int32_t *ipiv = reinterpret_cast<int32_t *>(base + off_ipiv);
  int32_t *info = reinterpret_cast<int32_t *>(base + off_info);
  posit_problem *desc = reinterpret_cast<posit_problem *>(base + off_desc);
  void *ws = base + off_ws;

  std::vector<posit_problem> wp((size_t)count);
  size_t w = 0, ip = 0;
  for (size_t i = 0; i < hp.size(); ++i) {
    const posit_problem &q = hp[i];
    posit_problem &r = wp[i];
    r = q;
    const int64_t n = q.n, ld = n > 0 ? n : 1;
    r.lda = ld;
    r.ldb = ld;
    r.A = work + w;
    if (n > 0 && cudaMemcpy2DAsync(pristine + w, (size_t)n * 4, q.A, (size_t)q.lda * 4,
                                   (size_t)n * 4, (size_t)n, cudaMemcpyDeviceToDevice,
                                   stream) != cudaSuccess)
      return POSIT_ERR_CUDA;
    w += (size_t)n * n;
    r.B = q.nrhs > 0 ? work + w : nullptr;
    if (n > 0 && q.nrhs > 0 &&
        cudaMemcpy2DAsync(pristine + w, (size_t)n * 4, q.B, (size_t)q.ldb * 4, (size_t)n * 4,
                          (size_t)q.nrhs, cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
      return POSIT_ERR_CUDA;
    w += (size_t)n * q.nrhs;
    r.ipiv = ipiv + ip;
    ip += (size_t)n;
    r.info = info + i;
  }
  if (cudaMemcpyAsync(desc, wp.data(), sizeof(posit_problem) * (size_t)count,
                      cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return POSIT_ERR_CUDA;

  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return POSIT_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return POSIT_ERR_CUDA;
  }
  int found = -1;
  float found_ms = 0.0f;
  int status = POSIT_OK;
  for (int32_t c = 0; c < ncand && status == POSIT_OK; ++c) {
    float t_best = -1.0f;
    if (plan_ok(&cands[c])) {
      for (int32_t r = 0; r < reps; ++r) {
        if (cudaMemcpyAsync(work, pristine, words * 4, cudaMemcpyDeviceToDevice, stream) !=
                cudaSuccess ||
            cudaEventRecord(e0, stream) != cudaSuccess) {
          status = POSIT_ERR_CUDA;
          break;
        }
        const int st = batched_launch(desc, order, count, (int)max_n, (int)max_nrhs, cands[c], ws,
                                      stream);
        if (st != POSIT_OK) {  // e.g. more shared memory than a CTA may have
          cudaGetLastError();
          t_best = -1.0f;
          break;
        }
        float ms = 0.0f;
        if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          status = POSIT_ERR_CUDA;
          break;
        }
        if (t_best < 0.0f || ms < t_best) t_best = ms;
      }
    }
    if (times_ms) times_ms[c] = t_best;
    if (t_best >= 0.0f && (found < 0 || plan_less(cands[c], t_best, cands[found], found_ms))) {
      found = c;
      found_ms = t_best;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != POSIT_OK) return status;
  if (found < 0) return POSIT_ERR_CUDA;
  *best = cands[found];
  return cudaStreamSynchronize(stream) == cudaSuccess ? POSIT_OK : POSIT_ERR_CUDA;
}
