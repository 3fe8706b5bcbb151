// solve.cu -- Rgetrs and Rpotrs (Sec. 5.1: the factors solve A x = b for the
// error study), in the reference-BLAS trsm operation orders that LAPACK's
// dgetrs/dpotrs (and MPLAPACK's R versions) use.
//
// Two kinds of triangular solve occur:
//   * "wavefront": every unknown receives its updates in the order in which
//     the unknowns are solved -- forward with ascending k, or backward with
//     descending k (column-oriented trsm; also the dot-form forward solve with
//     ascending k).  x_i's last update needs x_{i-1} (in solve order), so the
//     solve is one dependent step per unknown at best: a division, a product
//     and a rounded subtraction.  trsv_pipe_kernel keeps that path in ONE warp
//     and moves everything else off it (below).
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

constexpr int ST = 256;        // threads per CTA (dot-form and swap kernels)
constexpr int NRHS_CHUNK = 8;  // right-hand sides per wavefront launch
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// Pipelined wavefront solve
//
// The unknowns are cut into blocks of PB = 32 rows (a warp, lane = row),
// numbered J = 0, 1, ... in solve order (descending rows for a backward
// solve).  Tile (I, J) holds the coefficients that block J's unknowns
// contribute to block I's rows.  One right-hand side is one pipeline of warps:
//   * the diagonal warp solves the blocks one after another.  While it solves
//     block J (32 steps: divide x_t, broadcast it by a shuffle, apply it to
//     the rows after t) it also brings block J+1 up to date: first with tile
//     (J+1, J-1) from the unknowns of block J-1 (known), then with tile
//     (J+1, J) as block J's unknowns become final -- two rounded
//     multiply-subtracts per step on a chain that is independent of the
//     diagonal one.  Its tiles are staged in shared memory by cp.async one
//     block ahead.
//   * helper warps bring every later block I up to date with tiles
//     (I, 0) .. (I, I-3), each tile as soon as the diagonal warp has
//     published that block's unknowns (a flag per block), and publish the
//     partial sums of block I (another flag) one block-time before the
//     diagonal warp needs them.
// Every unknown still receives its updates in solve order, one rounded
// multiply and one rounded subtract each, so the bits equal the sequential
// loops'.  Solved values and the helpers' partial sums live in B itself.
// Every wait is bounded: after about 2 s of global time a warp sets the error
// flag and all warps return.
// ---------------------------------------------------------------------------
constexpr int PB = 32;       // rows per block
constexpr int PWARPS = 4;    // warps per CTA
constexpr int PT = PB * PWARPS;

struct PipeArgs {
  const uint32_t *A;
  int64_t lda;
  uint32_t *B;       // right-hand side c0 (blockIdx.y adds the column)
  int64_t ldb;
  int64_t n;
  int trans;         // element (i, k) of the triangle at A[k + i*lda] instead of A[i + k*lda]
  int unit;          // unit diagonal (no division; also a template argument)
  int nblk;          // number of PB-row blocks
  int *flags;        // per right-hand side: solved[nblk], ready[nblk] (zeroed)
  int *err;
  const int32_t *abort_flag;  // skip the solve when *abort_flag != 0
};

__device__ __forceinline__ int ld_acquire_flag(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_flag(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Every lane waits (acquire) for *flag != 0.  Bounded: lane 0 looks at the
// error flag and the clock every 64 polls; false after about 2 s (the error
// flag is then set) or when another warp has given up.
__device__ bool warp_wait(const int *flag, int *err) {
  unsigned long long t0 = 0;
  for (unsigned polls = 1;; ++polls) {
    const int v = ld_acquire_flag(flag);
    if (__all_sync(0xFFFFFFFFu, v != 0)) return true;
    if ((polls & 63u) == 0u) {
      int stop = 0;
      if ((threadIdx.x & 31) == 0) {
        if (*(volatile int *)err) {
          stop = 1;
        } else {
          const unsigned long long now = global_ns();
          if (t0 == 0) {
            t0 = now;
          } else if (now - t0 > kWaitNs) {
            atomicExch(err, 1);
            stop = 1;
          }
        }
      }
      if (__shfl_sync(0xFFFFFFFFu, stop, 0)) return false;
    }
    __nanosleep(32);
  }
}

// The warp's rows have been stored: make them visible, then raise the flag.
__device__ __forceinline__ void warp_publish(int *flag) {
  __threadfence();
  __syncwarp();
  if ((threadIdx.x & 31) == 0) st_release_flag(flag, 1);
}

// First row of block J (solve order) and its row count.
template <bool BW>
__device__ __forceinline__ int64_t pipe_row0(int J, int nblk) {
  return (int64_t)(BW ? nblk - 1 - J : J) * PB;
}

// Address of element (i, k) of the triangle (i, k < n).
__device__ __forceinline__ const uint32_t *pipe_elem(const PipeArgs &a, int64_t i, int64_t k) {
  return a.trans ? a.A + k + i * a.lda : a.A + i + k * a.lda;
}

__device__ __forceinline__ void cp_async4(uint32_t *dst, const uint32_t *src, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}

// Stage tile (rows of block I, columns of block J) as T[t][lane] (t = column
// within block J, lane = row within block I); entries outside the matrix,
// or of a block index outside [0, nblk), are zero.
template <bool BW>
__device__ __forceinline__ void stage_tile(const PipeArgs &a, uint32_t *T, int I, int J) {
  const int lane = threadIdx.x & 31;
  const bool blocks_ok = I >= 0 && I < a.nblk && J >= 0 && J < a.nblk;
  const int64_t r = blocks_ok ? pipe_row0<BW>(I, a.nblk) + lane : 0;
  const int64_t c0 = blocks_ok ? pipe_row0<BW>(J, a.nblk) : 0;
#pragma unroll 8
  for (int t = 0; t < PB; ++t) {
    const bool ok = blocks_ok && r < a.n && c0 + t < a.n;
    cp_async4(T + t * PB + lane, ok ? pipe_elem(a, r, c0 + t) : a.A, ok);
  }
}

// x_r of block J for this lane (zero for rows past n).
__device__ __forceinline__ pz load_x(const uint32_t *b, int64_t row0, int64_t n) {
  const int64_t r = row0 + (threadIdx.x & 31);
  return r < n ? pz_decode(__ldcg(b + r)) : pz_zero();
}

__device__ __forceinline__ void store_x(uint32_t *b, int64_t row0, int64_t n, pz x) {
  const int64_t r = row0 + (threadIdx.x & 31);
  if (r < n) b[r] = pz_to_bits(x);
}

__device__ __forceinline__ pz shfl_pz(pz v, int src) {
  return pz{__shfl_sync(0xFFFFFFFFu, v.s, src), __shfl_sync(0xFFFFFFFFu, v.m, src)};
}

// x - a * y with a given as a word
__device__ __forceinline__ pz msub(pz x, uint32_t aw, pz y) {
  return pz_sub(x, pz_mul(pz_decode(aw), y));
}

// ---- in-band fast path -----------------------------------------------------
// While every product of a chain has operands that are zero or of scale in
// [-40, 40], and the chain starts from a value of scale within [-80, 80], the
// chain's values stay multiples of 2^-107 below 2^89 (the bound argument of
// the Rgemm kernel), so no rounding needs the test for regimes of 28 or more
// bits.  The straight-line forms below give the same bits as the general
// ones there.

// A word that is zero or has its scale in [-40, 40]: |x| in [2^-40, 2^41).
__device__ __forceinline__ bool word_band(uint32_t w) {
  const uint32_t a = (int)w < 0 ? 0u - w : w;
  return w == 0u || a - 0x00100000u < 0x7FF20000u - 0x00100000u;
}

__device__ __forceinline__ bool pz_band(pz v, int lim) {
  return pz_is_zero(v) || (v.s >= -lim && v.s <= lim);
}

// pz_decode of a word that is not NaR, without branches.
__device__ __forceinline__ pz decode_band(uint32_t p) {
  const uint32_t sign = p & 0x80000000u;
  const uint32_t a = sign ? 0u - p : p;
  const uint32_t x = a << 1;
  const uint32_t first = x >> 31;
  const int m = __clz(first ? ~x : x);
  const int k = first ? m - 1 : -m;
  const uint32_t rest = (x << (m & 31)) << 1;
  const int e = (int)(rest >> 30);
  const uint32_t mag = (1u << 30) | ((rest << 2) >> 2);
  return pz{p ? 4 * k + e : PZ_SZERO, p ? (sign | mag) : 0u};
}

// Round to nearest even for a scale of at most 107 in magnitude (or a zero
// significand): pz_round without the test for the long regimes, the
// constants computed from the scale instead of read from a table (a single
// warp's dependency chain would wait for every bank conflict of the
// per-lane table rows).
__device__ __forceinline__ pz round_band(uint32_t sign, int S, uint32_t X) {
  const int km = (S >> 2) ^ (S >> 31);
  const uint32_t q = min((uint32_t)km + 3u, 30u);
  const uint32_t lsb = (X >> q) & 1u;
  uint32_t r = X + ((1u << (q - 1)) - 1u) + lsb;
  r &= ~((1u << q) - 1u);
  const uint32_t c = r >> 31;
  return pz{S + (int)c, sign | (r >> c)};
}

// msub for in-band operands and a chain value as above.
__device__ __forceinline__ pz msub_band(pz x, uint32_t aw, pz y) {
  uint32_t sg, X0, jam, Xs;
  int S, Ss;
  pz_mul_parts(decode_band(aw), y, sg, S, X0, jam);
  const pz p = round_band(sg, S, X0 | jam);
  pz_add_exact_inband(x, pz{p.s, p.m ^ 0x80000000u}, sg, Ss, Xs);
  return round_band(sg, Ss, Xs);
}

// floor(2^62 / B) for the significand B of a divisor d (B in [2^30, 2^31)),
// computed once per divisor off the dependency chain.
__device__ __forceinline__ uint64_t recip62(pz d) {
  const uint32_t B = max(d.m & 0x7FFFFFFFu, 1u << 30);
  return (1ull << 62) / (uint64_t)B;
}

// x / d with R = recip62(d), for d nonzero and in band and x zero or a chain
// value as above.  floor(A 2^31 / B) from the reciprocal: with R = 2^62 / B
// - e (0 <= e < 1) and A < 2^31, floor(A R / 2^31) is the quotient q or
// q - 1, so one correction from the exact remainder gives q and the
// inexact bit -- what pz_sig_div gives -- then the steps of pz_div with the
// in-band rounding.  Exact whenever the result's scale is in [-40, 40];
// callers check that and take pz_div otherwise.
__device__ __forceinline__ pz div_recip(pz x, pz d, uint64_t R) {
  const uint32_t A = x.m & 0x7FFFFFFFu, B = d.m & 0x7FFFFFFFu;
  uint64_t q = ((uint64_t)A * R) >> 31;
  int64_t rem = (int64_t)((uint64_t)A << 31) - (int64_t)(q * B);
  const bool up = rem >= (int64_t)B;
  q = up ? q + 1u : q;
  rem = up ? rem - (int64_t)B : rem;
  const uint32_t qq = (uint32_t)q, jam = rem != 0;
  const uint32_t top = qq >> 31;
  const uint32_t X = top ? ((qq >> 1) | (qq & 1u) | jam) : (qq | jam);
  const int S = x.s - d.s - (int)(top ^ 1u);
  return round_band((x.m ^ d.m) & 0x80000000u, S, X);
}

// Shared memory of one CTA: the diagonal warp's tiles (D, C, S for three
// blocks: the one being solved, the next, and the one after it, which is
// staged while the current one is solved; used by the pipeline's first CTA
// only) and two tiles per helper warp.
constexpr int kTileWords = PB * PB;
constexpr int kDiagBufs = 3;
constexpr size_t kPipeSmem = (kDiagBufs * 3 + PWARPS * 2) * kTileWords * sizeof(uint32_t);

// Column t of the three tiles the diagonal warp uses for block J (D = (J, J),
// C = (J+1, J-1), S = (J+1, J)), one cp.async per lane and tile.
template <bool BW>
__device__ __forceinline__ void stage_diag_column(const PipeArgs &a, uint32_t *buf, int J,
                                                  int t) {
  const int lane = threadIdx.x & 31;
  const int nb = a.nblk;
  const int I[3] = {J, J + 1, J + 1};
  const int C[3] = {J, J - 1, J};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const bool blocks_ok = I[q] >= 0 && I[q] < nb && C[q] >= 0 && C[q] < nb;
    const int64_t r = pipe_row0<BW>(blocks_ok ? I[q] : 0, nb) + lane;
    const int64_t c = pipe_row0<BW>(blocks_ok ? C[q] : 0, nb) + t;
    const bool ok = blocks_ok && r < a.n && c < a.n;
    cp_async4(buf + q * kTileWords + t * PB + lane, ok ? pipe_elem(a, r, c) : a.A, ok);
  }
}

// (PT, 1): ptxas keeps enough registers for the three chains of a step to
// overlap; with its default budget they run one after another (measured
// 953 against 651 cycles per step in a one-warp probe of the step).
template <bool BW, bool UNIT>
__global__ void __launch_bounds__(PT, 1) trsv_pipe_kernel(PipeArgs a) {
  extern __shared__ __align__(16) uint32_t psmem[];
  const int lane = threadIdx.x & 31;
  const int wl = threadIdx.x >> 5;                 // warp within the CTA
  const int w = blockIdx.x * PWARPS + wl;          // warp within the pipeline
  const int nblk = a.nblk;
  uint32_t *b = a.B + (int64_t)blockIdx.y * a.ldb;
  int *solved = a.flags + (int64_t)blockIdx.y * 2 * nblk;
  int *ready = solved + nblk;  // 1: partial sums published from a clean chain, 2: not clean
  if (a.abort_flag && *(volatile const int32_t *)a.abort_flag != 0) return;
  const unsigned FULL = 0xFFFFFFFFu;

  if (w == 0) {
    // ------------------------------------------------ the diagonal warp
    // Each step is straight-line code (every lane computes, selects keep
    // the lanes that apply), so the diagonal chain (divide, broadcast,
    // multiply-subtract), the chain of block J+1 and the staging of block
    // J+2's tiles are interleaved by the compiler.  A block runs on the
    // in-band forms when its tiles, the unknowns it uses and both chains
    // qualify; a step whose new unknown leaves the band is redone on the
    // general forms, as is the rest of that block.
    uint32_t *tiles = psmem;  // [kDiagBufs][3][kTileWords]
    for (int J0 = 0; J0 < 2; ++J0) {
      for (int t = 0; t < PB; ++t) stage_diag_column<BW>(a, tiles + J0 * 3 * kTileWords, J0, t);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    pz x = load_x(b, pipe_row0<BW>(0, nblk), a.n);
    pz xn = nblk > 1 ? load_x(b, pipe_row0<BW>(1, nblk), a.n) : pz_zero();
    pz xprev = pz_zero();
    // the chains of x (block J) and xn (block J+1) are clean
    bool cx = __all_sync(FULL, pz_band(x, 80)), cn = __all_sync(FULL, pz_band(xn, 80));
    bool ok = true;
    for (int J = 0; J < nblk && ok; ++J) {
      asm volatile("cp.async.wait_group 1;" ::: "memory");  // block J's tiles are in
      __syncwarp();
      const uint32_t *D = tiles + (J % kDiagBufs) * 3 * kTileWords;
      const uint32_t *Cc = D + kTileWords, *Sx = D + 2 * kTileWords;
      uint32_t *nxt = tiles + ((J + 2) % kDiagBufs) * 3 * kTileWords;
      const int64_t row0 = pipe_row0<BW>(J, nblk);
      const int nr = (int)min64(PB, a.n - row0);
      if (lane >= nr) x = pz_zero();
      const pz dl = pz_decode(D[lane * PB + lane]);
      const uint64_t rl = UNIT ? 0ull : recip62(dl);
      bool tok = pz_band(xprev, 40) && (UNIT || lane >= nr || (!pz_is_zero(dl)));
#pragma unroll 8
      for (int t = 0; t < PB; ++t)
        tok &= word_band(D[t * PB + lane]) && word_band(Cc[t * PB + lane]) &&
               word_band(Sx[t * PB + lane]);
      tok = __all_sync(FULL, tok);
      bool fast = cx && cn && tok;
      bool xn_clean = cn && tok;  // every product xn receives in this block is in band
      pz xnn = pz_zero();
      bool cnn = false;
      for (int half = 0; half < 2; ++half) {
        if (half == 1 && J + 2 < nblk) {
          // block J+2's partial sums, long published by its helper
          if (!warp_wait(&ready[J + 2], a.err)) { ok = false; break; }
          cnn = __ldcg(&ready[J + 2]) == 1;
          xnn = load_x(b, pipe_row0<BW>(J + 2, nblk), a.n);
        }
        const uint32_t *T = half ? Sx : Cc;
        const int s_end = (half + 1) * (PB / 2);
        int s = half * (PB / 2);
        // Each step: block J+1 gets two links on unknowns that are final
        // before the step begins (so their shuffles do not wait for it):
        // ua, ub (solve order) of block J-1 in the first half; of block J in
        // the second half, one step behind (ua = -1 at its first step is a
        // multiply by zero, and block J's last unknown follows the loop).
        if (fast) {
#pragma unroll 1
          for (; s < s_end; ++s) {
            const int t = BW ? PB - 1 - s : s;
            const int ua = half ? 2 * s - 33 : 2 * s, ub = ua + 1;
            const int ta = BW ? PB - 1 - max(ua, 0) : max(ua, 0), tb = BW ? PB - 1 - ub : ub;
            const pz src = half ? x : xprev;
            pz ya = shfl_pz(src, ta);
            const pz yb = shfl_pz(src, tb);
            if (ua < 0) ya = pz_zero();
            pz xs = x;
            if (!UNIT) {
              const pz q = div_recip(x, dl, rl);
              const bool dv = lane == t && t < nr;
              xs = pz{dv ? q.s : x.s, dv ? q.m : x.m};
            }
            const pz xt = shfl_pz(xs, t);
            const pz r = msub_band(xs, D[t * PB + lane], xt);
            const bool up = (BW ? lane < t : lane > t) && lane < nr;
            xs = pz{up ? r.s : xs.s, up ? r.m : xs.m};
            pz xns = msub_band(xn, T[ta * PB + lane], ya);
            xns = msub_band(xns, T[tb * PB + lane], yb);
            if (!pz_band(xt, 40)) break;  // the same on every lane: redo this step below
            x = xs;
            xn = xns;
            stage_diag_column<BW>(a, nxt, J + 2, s);
          }
          if (s < s_end) fast = false;
        }
#pragma unroll 1
        for (; s < s_end; ++s) {
          const int t = BW ? PB - 1 - s : s;
          const int ua = half ? 2 * s - 33 : 2 * s, ub = ua + 1;
          const int ta = BW ? PB - 1 - max(ua, 0) : max(ua, 0), tb = BW ? PB - 1 - ub : ub;
          const pz src = half ? x : xprev;
          pz ya = shfl_pz(src, ta);
          const pz yb = shfl_pz(src, tb);
          if (ua < 0) ya = pz_zero();
          if (!UNIT) {
            const pz q = pz_div_inline(x, dl);
            const bool dv = lane == t && t < nr;
            x = pz{dv ? q.s : x.s, dv ? q.m : x.m};
          }
          const pz xt = shfl_pz(x, t);
          xn_clean = xn_clean && pz_band(xt, 40);
          const pz r = msub(x, D[t * PB + lane], xt);
          const bool up = (BW ? lane < t : lane > t) && lane < nr;
          x = pz{up ? r.s : x.s, up ? r.m : x.m};
          xn = msub(xn, T[ta * PB + lane], ya);
          xn = msub(xn, T[tb * PB + lane], yb);
          stage_diag_column<BW>(a, nxt, J + 2, s);
        }
        if (half == 1) {  // block J's last unknown into block J+1
          const int tl = BW ? 0 : PB - 1;
          const pz yl = shfl_pz(x, tl);
          xn = fast ? msub_band(xn, Sx[tl * PB + lane], yl) : msub(xn, Sx[tl * PB + lane], yl);
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      if (!ok) break;
      store_x(b, row0, a.n, x);
      warp_publish(&solved[J]);
      xprev = x;
      x = xn;
      cx = xn_clean;
      xn = xnn;
      cn = cnn;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    return;
  }

  // ---------------------------------------------------- helper warps
  // Helper h brings blocks I = 2 + h, 2 + h + H, ... up to date with tiles
  // (I, J) for J <= I - 3, in J order, two blocks at a time (two independent
  // chains per lane); partial sums stay in B's rows of I.  A tile whose words
  // and unknowns are all in band, applied to clean chains, runs on the
  // in-band forms.  Bit k of `dirty` marks the helper's k-th block as not
  // clean (blocks past the 32nd are treated as not clean).
  uint32_t *ht = psmem + (kDiagBufs * 3 + wl * 2) * kTileWords;  // [2][kTileWords]
  const int H = gridDim.x * PWARPS - 1;
  const int h = w - 1;
  int Ilast = -1;
  for (int I = 2 + h; I < nblk; I += H) Ilast = I;
  if (Ilast < 0) return;
  unsigned dirty = 0;
  for (int I = 2 + h, k = 0; I <= Ilast; I += H, ++k) {
    const bool c = __all_sync(FULL, pz_band(load_x(b, pipe_row0<BW>(I, nblk), a.n), 80));
    if (!c || k >= 32) dirty |= k < 32 ? (1u << k) : 0u;
  }
  auto is_clean = [&](int I) {
    const int k = (I - 2 - h) / H;
    return k < 32 && !((dirty >> k) & 1u);
  };
  if (h == 0) {  // block 2 enters the window unchanged
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release_flag(&ready[2], is_clean(2) ? 1 : 2);
  }
  for (int J = 0; J <= Ilast - 3; ++J) {
    const int64_t c0 = pipe_row0<BW>(J, nblk);
    int I = 2 + h;
    while (I < J + 3) I += H;
    bool waited = false;
    for (; I <= Ilast; I += 2 * H) {
      const int I2 = I + H <= Ilast ? I + H : -1;
      // tiles staged and partial sums loaded before the wait for block J
      stage_tile<BW>(a, ht, I, J);
      stage_tile<BW>(a, ht + kTileWords, I2, J);
      asm volatile("cp.async.commit_group;" ::: "memory");
      const int64_t r1 = pipe_row0<BW>(I, nblk);
      const int64_t r2 = I2 >= 0 ? pipe_row0<BW>(I2, nblk) : r1;
      pz x1 = load_x(b, r1, a.n);
      pz x2 = load_x(b, r2, a.n);
      if (!waited) {
        if (!warp_wait(&solved[J], a.err)) {
          asm volatile("cp.async.wait_group 0;" ::: "memory");
          return;
        }
        waited = true;
      }
      const pz xj = load_x(b, c0, a.n);
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncwarp();
      bool ok1 = pz_band(xj, 40), ok2 = ok1;
#pragma unroll 8
      for (int t = 0; t < PB; ++t) {
        ok1 &= word_band(ht[t * PB + lane]);
        ok2 &= word_band(ht[kTileWords + t * PB + lane]);
      }
      ok1 = __all_sync(FULL, ok1) && is_clean(I);
      ok2 = __all_sync(FULL, ok2) && (I2 < 0 || is_clean(I2));
      if (ok1 && ok2) {
#pragma unroll 2
        for (int s = 0; s < PB; ++s) {
          const int t = BW ? PB - 1 - s : s;
          const pz y = shfl_pz(xj, t);
          x1 = msub_band(x1, ht[t * PB + lane], y);
          x2 = msub_band(x2, ht[kTileWords + t * PB + lane], y);
        }
      } else {
#pragma unroll 2
        for (int s = 0; s < PB; ++s) {
          const int t = BW ? PB - 1 - s : s;
          const pz y = shfl_pz(xj, t);
          x1 = msub(x1, ht[t * PB + lane], y);
          x2 = msub(x2, ht[kTileWords + t * PB + lane], y);
        }
        const int k1 = (I - 2 - h) / H;
        if (!ok1 && k1 < 32) dirty |= 1u << k1;
        if (I2 >= 0 && !ok2) {
          const int k2 = (I2 - 2 - h) / H;
          if (k2 < 32) dirty |= 1u << k2;
        }
      }
      store_x(b, r1, a.n, x1);
      if (I2 >= 0) store_x(b, r2, a.n, x2);
      __threadfence();
      __syncwarp();  // the tiles are read before the next pair restages them
      if (lane == 0) {
        if (J == I - 3) st_release_flag(&ready[I], is_clean(I) ? 1 : 2);
        if (I2 >= 0 && J == I2 - 3) st_release_flag(&ready[I2], is_clean(I2) ? 1 : 2);
      }
    }
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


// Scratch of one wavefront launch: the error flag, then two flags per block
// for each of up to NRHS_CHUNK right-hand sides.
constexpr size_t kPipeHead = 256;

size_t pipe_flag_bytes(int64_t n) { return 2 * (size_t)ceil_div(n, PB) * sizeof(int); }

// One wavefront solve (see trsv_pipe_kernel) of the nrhs columns of B, in
// launches of up to NRHS_CHUNK pipelines (one per right-hand side).
int trsv_pipe(const uint32_t *A, int64_t lda, int trans, int backward, int unit, uint32_t *B,
              int64_t ldb, int64_t n, int64_t nrhs, void *scratch, size_t scratch_bytes,
              const Limits &l, cudaStream_t stream, const int32_t *abort_flag = nullptr) {
  const int64_t nblk = ceil_div(n, PB);
  const size_t per_rhs = pipe_flag_bytes(n);
  if (nblk > (1 << 30) || scratch_bytes < kPipeHead + per_rhs) return POSIT_ERR_DEVICE;
  const void *fn = backward ? (unit ? (const void *)trsv_pipe_kernel<true, true>
                                    : (const void *)trsv_pipe_kernel<true, false>)
                            : (unit ? (const void *)trsv_pipe_kernel<false, true>
                                    : (const void *)trsv_pipe_kernel<false, false>);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPipeSmem) !=
      cudaSuccess)
    return POSIT_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PT, kPipeSmem) != cudaSuccess ||
      per_sm < 1)
    return POSIT_ERR_CUDA;
  const int64_t resident = (int64_t)per_sm * l.sms;
  // one block per helper warp keeps the helpers ahead of the diagonal warp;
  // with fewer co-resident warps each helper takes several blocks (slower)
  const int64_t helpers = max64(3, nblk - 2);
  const int64_t gx = min64(ceil_div(helpers + 1, PWARPS), resident);
  int64_t chunk = min64(NRHS_CHUNK, (int64_t)((scratch_bytes - kPipeHead) / per_rhs));
  chunk = max64(1, min64(chunk, resident / gx));
  for (int64_t c0 = 0; c0 < nrhs; c0 += chunk) {
    const int64_t nc = min64(chunk, nrhs - c0);
    if (cudaMemsetAsync(scratch, 0, kPipeHead + per_rhs * nc, stream) != cudaSuccess)
      return POSIT_ERR_CUDA;
    PipeArgs pa;
    pa.A = A; pa.lda = lda; pa.B = B + c0 * ldb; pa.ldb = ldb; pa.n = n;
    pa.trans = trans; pa.unit = unit; pa.nblk = (int)nblk;
    pa.err = static_cast<int *>(scratch);
    pa.flags = reinterpret_cast<int *>(static_cast<char *>(scratch) + kPipeHead);
    pa.abort_flag = abort_flag;
    void *args[] = {&pa};
    if (cudaLaunchCooperativeKernel(fn, dim3((unsigned)gx, (unsigned)nc), dim3(PT), args,
                                    kPipeSmem, stream) != cudaSuccess)
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

size_t solve_scratch_bytes(int64_t n) { return kPipeHead + pipe_flag_bytes(n) * NRHS_CHUNK; }

int getrs_run(bool trans, int64_t n, int64_t nrhs, const uint32_t *A, int64_t lda,
              const int32_t *ipiv, uint32_t *B, int64_t ldb, void *scratch, size_t scratch_bytes,
              cudaStream_t stream) {
  Limits l;
  int st = limits(l);
  if (st) return st;
  if (!trans) {
    if ((st = laswp_vec(B, ldb, n, nrhs, ipiv, false, l, stream))) return st;
    // L y = b (unit lower): ascending, column order
    if ((st = trsv_pipe(A, lda, 0, 0, 1, B, ldb, n, nrhs, scratch, scratch_bytes, l, stream)))
      return st;
    // U x = y: descending, column order, divide by u_ii
    return trsv_pipe(A, lda, 0, 1, 0, B, ldb, n, nrhs, scratch, scratch_bytes, l, stream);
  }
  // U^T y = b: ascending dot form (a wavefront over U accessed transposed)
  if ((st = trsv_pipe(A, lda, 1, 0, 0, B, ldb, n, nrhs, scratch, scratch_bytes, l, stream)))
    return st;
  // L^T z = y, unit: dot form, k ascending -- serial chain
  if ((st = trsv_dot_backward(A, lda, 1, B, ldb, n, nrhs, l, stream))) return st;
  return laswp_vec(B, ldb, n, nrhs, ipiv, true, l, stream);
}

int potrs_run_guarded(bool upper, int64_t n, int64_t nrhs, const uint32_t *A, int64_t lda,
                      uint32_t *B, int64_t ldb, const int32_t *abort_flag, void *scratch,
                      size_t scratch_bytes, cudaStream_t stream) {
  Limits l;
  int st = limits(l);
  if (st) return st;
  if (!upper) {
    // L y = b: ascending, then divide
    if ((st = trsv_pipe(A, lda, 0, 0, 0, B, ldb, n, nrhs, scratch, scratch_bytes, l, stream,
                        abort_flag)))
      return st;
    // L^T x = y: dot form, k ascending -- serial chain
    return trsv_dot_backward(A, lda, 0, B, ldb, n, nrhs, l, stream, abort_flag);
  }
  // U^T y = b: ascending dot form
  if ((st = trsv_pipe(A, lda, 1, 0, 0, B, ldb, n, nrhs, scratch, scratch_bytes, l, stream,
                      abort_flag)))
    return st;
  // U x = y: descending, column order
  return trsv_pipe(A, lda, 0, 1, 0, B, ldb, n, nrhs, scratch, scratch_bytes, l, stream,
                   abort_flag);
}

int potrs_run(bool upper, int64_t n, int64_t nrhs, const uint32_t *A, int64_t lda, uint32_t *B,
              int64_t ldb, void *scratch, size_t scratch_bytes, cudaStream_t stream) {
  return potrs_run_guarded(upper, n, nrhs, A, lda, B, ldb, nullptr, scratch, scratch_bytes,
                           stream);
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
  const size_t bytes = solve_scratch_bytes(n);
  if (cudaMallocAsync(&scratch, bytes, stream) != cudaSuccess) {
    cudaGetLastError();
    return POSIT_ERR_ALLOC;
  }
  int st = getrs_run(is_trans(trans), n, nrhs, A, lda, ipiv, B, ldb, scratch, bytes, stream);
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
  const size_t bytes = solve_scratch_bytes(n);
  if (cudaMallocAsync(&scratch, bytes, stream) != cudaSuccess) {
    cudaGetLastError();
    return POSIT_ERR_ALLOC;
  }
  int st = potrs_run(is_upper(uplo), n, nrhs, A, lda, B, ldb, scratch, bytes, stream);
  cudaFreeAsync(scratch, stream);
  return st;
}
