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
//     and a rounded subtraction.  trsv_pipe_kernel keeps that path in one
//     warp and moves everything else off it (below).
//   * "dot-form backward": x_i = (b_i - sum_{k = i+1 .. n-1, ascending}
//     a_ki x_k) / a_ii, i descending (reference trsm Left-Lower-Transpose).
//     x_i's first subtraction needs x_{i+1}, the last unknown to finish, so
//     the n(n-1)/2 subtractions form one serial chain per right-hand side.
//     trsv_dot_backward_kernel computes the products of each row in parallel
//     and runs the chain of rounded additions in one thread, in the signed
//     chain form of chain.cuh (about half the instructions of a general
//     addition per link).
//
// Row swaps (ipiv, LAPACK convention) are applied by a one-CTA-per-column
// kernel on a shared-memory copy of the column.
#include <cstdlib>

#include "internal.cuh"
#include "chain.cuh"

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
//   * the diagonal warp solves the blocks one after another (32 steps:
//     divide x_t, broadcast it by a shuffle, apply it to the rows after t)
//     and posts every unknown, as soon as it is final, in shared memory;
//   * KS streaming warps (same CTA): while block J is solved, streaming warp
//     k applies tile (J+k, J) to block J+k as block J's unknowns appear, and
//     passes block J+k's sums on to warp k-1 (warp 1: to the diagonal warp,
//     which solves block J+1 next; warp 1 also writes block J's unknowns to
//     B).  Each warp thus handles one tile per block time and keeps pace
//     with the diagonal warp; warp KS takes its block's sums from
//   * helper warps (the other CTAs), which bring every later block I up to
//     date with tiles (I, 0) .. (I, I-KS-1), each tile as soon as its
//     block's unknowns are published (a flag per block), and publish block
//     I's partial sums (another flag).  The streaming warps absorb the
//     helpers' lag: warp KS may start a tile late and catch up, since the
//     unknowns it needs are already posted.
// Every unknown still receives its updates in solve order, one rounded
// multiply and one rounded subtract each, so the bits equal the sequential
// loops'.  Solved values and the helpers' partial sums live in B itself.
// Every wait is bounded: after about 2 s of global time a warp sets the error
// flag and all warps return.
// ---------------------------------------------------------------------------
constexpr int PB = 32;       // rows per block
constexpr int PWARPS = 4;    // warps per CTA
constexpr int PT = PB * PWARPS;
constexpr int KS = PWARPS - 1;   // streaming warps: the first CTA but its diagonal warp
constexpr int kSlotBufs = KS + 1;

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

// pz_to_bits of a rounded value that is not NaR, without branches: both
// regime forms are built and selected (the clamps change nothing for the
// regimes of rounded values, k in [-30, 30]; a zero's arbitrary scale is
// overridden).
__device__ __forceinline__ uint32_t bits_band(pz a) {
  const int k = a.s >> 2;
  const uint32_t body = ((uint32_t)(a.s & 3) << 27) | ((a.m & 0x3FFFFFFFu) >> 3);
  const uint32_t kp = (uint32_t)min(max(k, 0), 30), kn = (uint32_t)min(max(-1 - k, 0), 29);
  const uint32_t pos = (0x7FFFFFFFu ^ (0x7FFFFFFFu >> (kp + 1u))) | (body >> kp);
  const uint32_t neg = (1u << (29u - kn)) | (body >> kn);
  const uint32_t pay = k >= 0 ? pos : neg;
  const uint32_t w = (a.m >> 31) ? (0u - pay) : pay;
  return pz_is_zero(a) ? 0u : w;
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

// Shared memory of one CTA.  The pipeline's first CTA holds the diagonal
// warp's tiles D = (J, J) and each streaming warp's tiles (J+k, J), each for
// three blocks (in use, next, being staged); in the other CTAs every helper
// warp stages two tiles.
constexpr int kTileWords = PB * PB;
constexpr int kBufs = 3;
constexpr int kPipeTiles = kBufs * (1 + KS) > 2 * PWARPS ? kBufs * (1 + KS) : 2 * PWARPS;
constexpr size_t kPipeSmem = (size_t)kPipeTiles * kTileWords * sizeof(uint32_t);
// Dynamic shared memory requested per CTA: more than the tiles need, so that
// at most two CTAs share an SM (with up to four, a pipeline's first CTA shares
// its SM's schedulers with helper CTAs: 8 right-hand sides at n = 8192 took
// 12.6 ms against 9.4 with two and 14.1 with one, when too few helpers fit).
constexpr size_t kPipeLaunchSmem = 76 * 1024;
static_assert(kPipeLaunchSmem >= kPipeSmem, "the launch covers the tiles");

// The first CTA's exchange (static shared memory).  slot[J % kSlotBufs][s] =
// (J * 64 + s + 1) << 32 | word of block J's unknown of step s: one 64-bit
// store carries the value and its tag, so the reader needs no fence; a
// buffer is rewritten KS + 1 blocks later, after every streaming warp has
// read it.  xh[I & 1][k] holds block I's sums from streaming warp k (hand[k]
// = I once written; taken[k] = I once its reader has copied them, so that
// the buffer can be reused for block I + 2).
struct PipeExchange {
  unsigned long long slot[kSlotBufs][PB];
  pz xh[2][KS + 1][PB];
  int clean[2][KS + 1];  // the chain that produced xh[..][k] stayed in band
  int hand[KS + 1];
  int taken[KS + 1];
};

// Bounded wait of a warp until `cond()` holds (shared-memory polls); false
// after about 2 s (error flag set) or when another warp has given up.
template <class Cond>
__device__ bool warp_spin(Cond cond, int *err) {
  unsigned long long t0 = 0;
  for (unsigned polls = 1;; ++polls) {
    if (__all_sync(0xFFFFFFFFu, cond())) return true;
    if ((polls & 255u) == 0u) {
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
  }
}

// (PT, 1): ptxas keeps enough registers for the chains of a step to
// overlap; with its default budget they run one after another (measured
// 953 against 651 cycles per step in a one-warp probe of the step).
template <bool BW, bool UNIT>
__global__ void __launch_bounds__(PT, 1) trsv_pipe_kernel(PipeArgs a) {
  extern __shared__ __align__(16) uint32_t psmem[];
  __shared__ PipeExchange ex;
  const int lane = threadIdx.x & 31;
  const int wl = threadIdx.x >> 5;  // warp within the CTA
  const int nblk = a.nblk;
  uint32_t *b = a.B + (int64_t)blockIdx.y * a.ldb;
  int *solved = a.flags + (int64_t)blockIdx.y * 2 * nblk;
  int *ready = solved + nblk;  // 1: partial sums published from a clean chain, 2: not clean
  const unsigned FULL = 0xFFFFFFFFu;
  if (a.abort_flag && *(volatile const int32_t *)a.abort_flag != 0) return;
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < kSlotBufs * PB; i += PT) (&ex.slot[0][0])[i] = 0ull;
    if (threadIdx.x <= KS) {
      ex.hand[threadIdx.x] = -1;
      ex.taken[threadIdx.x] = -1;
    }
  }
  __syncthreads();

  if (blockIdx.x == 0 && wl == 0) {
    // ------------------------------------------------ the diagonal warp
    // Solves the blocks one after another: per step, divide x_t, broadcast
    // it, apply it to the rows after t -- straight-line code (every lane
    // computes, selects keep the lanes that apply) -- and post x_t for the
    // streaming warps.  A block runs on the in-band forms while its tile,
    // its chain and the new unknowns qualify; a step whose unknown leaves
    // the band is redone on the general forms, as is the rest of that block.
    uint32_t *dt = psmem;  // [kBufs][kTileWords]: D of three blocks
    stage_tile<BW>(a, dt, 0, 0);
    asm volatile("cp.async.commit_group;" ::: "memory");
    stage_tile<BW>(a, dt + kTileWords, 1, 1);
    asm volatile("cp.async.commit_group;" ::: "memory");
    pz x = load_x(b, pipe_row0<BW>(0, nblk), a.n);
    bool cx = __all_sync(FULL, pz_band(x, 80));
    for (int J = 0; J < nblk; ++J) {
      if (J > 0) {  // block J's sums through tile J-1, from streaming warp 1
        if (!warp_spin([&] { return *(volatile int *)&ex.hand[1] >= J; }, a.err)) break;
        x = ex.xh[J & 1][1][lane];
        cx = *(volatile int *)&ex.clean[J & 1][1] != 0;
        __syncwarp();
        if (lane == 0) *(volatile int *)&ex.taken[1] = J;
      }
      stage_tile<BW>(a, dt + ((J + 2) % kBufs) * kTileWords, J + 2, J + 2);
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_group 1;" ::: "memory");
      __syncwarp();
      const uint32_t *D = dt + (J % kBufs) * kTileWords;
      unsigned long long *slot = ex.slot[J % kSlotBufs];
      const unsigned long long tag = (unsigned long long)(J * 64) << 32;
      const int64_t row0 = pipe_row0<BW>(J, nblk);
      const int nr = (int)min64(PB, a.n - row0);
      if (lane >= nr) x = pz_zero();
      const pz dl = pz_decode(D[lane * PB + lane]);
      const uint64_t rl = UNIT ? 0ull : recip62(dl);
      bool tok = UNIT || lane >= nr || !pz_is_zero(dl);
#pragma unroll 8
      for (int t = 0; t < PB; ++t) tok &= word_band(D[t * PB + lane]);
      int s = 0;
      if (cx && __all_sync(FULL, tok)) {
#pragma unroll 1
        for (; s < PB; ++s) {
          const int t = BW ? PB - 1 - s : s;
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
          if (!pz_band(xt, 40)) break;  // the same on every lane: redo this step below
          x = xs;
          // every lane stores the same word (xt came from one lane): no
          // divergent branch on the step's path
          *(volatile unsigned long long *)&slot[s] =
              tag + ((unsigned long long)(s + 1) << 32) + bits_band(xt);
        }
      }
#pragma unroll 1
      for (; s < PB; ++s) {
        const int t = BW ? PB - 1 - s : s;
        if (!UNIT) {
          const pz q = pz_div_inline(x, dl);
          const bool dv = lane == t && t < nr;
          x = pz{dv ? q.s : x.s, dv ? q.m : x.m};
        }
        const pz xt = shfl_pz(x, t);
        const pz r = msub(x, D[t * PB + lane], xt);
        const bool up = (BW ? lane < t : lane > t) && lane < nr;
        x = pz{up ? r.s : x.s, up ? r.m : x.m};
        *(volatile unsigned long long *)&slot[s] =
            tag + ((unsigned long long)(s + 1) << 32) + pz_to_bits(xt);
      }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    return;
  }

  if (blockIdx.x == 0) {
    // ------------------------------------------------ streaming warp k
    // While the diagonal warp solves block J, applies tile (J+k, J) to block
    // J+k as block J's unknowns are posted.  Block J+k's sums through tile
    // J-1 come from streaming warp k+1 (warp KS: from the helpers; J = 0:
    // straight from B); its sums through tile J go to warp k-1 (warp 1: to
    // the diagonal warp).  Warp 1 also writes block J's unknowns to B and
    // raises `solved[J]` for the helpers.
    const int k = wl;
    uint32_t *st = psmem + (size_t)kBufs * k * kTileWords;  // [kBufs][kTileWords]
    stage_tile<BW>(a, st, k, 0);
    asm volatile("cp.async.commit_group;" ::: "memory");
    stage_tile<BW>(a, st + kTileWords, k + 1, 1);
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int J = 0; J < nblk; ++J) {
      const int I = J + k;
      const bool has = I < nblk;
      if (!has && k > 1) break;  // nothing left for this warp
      pz xn = pz_zero();
      bool clean = false;
      if (has) {
        if (J == 0) {
          xn = load_x(b, pipe_row0<BW>(I, nblk), a.n);
          clean = __all_sync(FULL, pz_band(xn, 80));
        } else if (k == KS) {
          if (!warp_wait(&ready[I], a.err)) break;
          clean = __ldcg(&ready[I]) == 1;
          xn = load_x(b, pipe_row0<BW>(I, nblk), a.n);
        } else {
          if (!warp_spin([&] { return *(volatile int *)&ex.hand[k + 1] >= I; }, a.err)) break;
          xn = ex.xh[I & 1][k + 1][lane];
          clean = *(volatile int *)&ex.clean[I & 1][k + 1] != 0;
          __syncwarp();
          if (lane == 0) *(volatile int *)&ex.taken[k + 1] = I;
        }
      }
      stage_tile<BW>(a, st + ((J + 2) % kBufs) * kTileWords, J + 2 + k, J + 2);
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_group 1;" ::: "memory");
      __syncwarp();
      const uint32_t *T = st + (J % kBufs) * kTileWords;
      bool tok = true;
#pragma unroll 8
      for (int t = 0; t < PB; ++t) tok &= word_band(T[t * PB + lane]);
      clean = clean && __all_sync(FULL, tok);
      const unsigned long long *slot = ex.slot[J % kSlotBufs];
      pz xcur = pz_zero();
      bool gave_up = false;
      // the unknowns in groups of SG: wait for the group's last one (they are
      // posted in order), form the group's products side by side, then run
      // its chain of subtractions -- a warp that runs behind the diagonal
      // warp catches up at the products' throughput, not one step's latency
      constexpr int SG = 8;
#pragma unroll 1
      for (int g = 0; g < PB; g += SG) {
        const unsigned long long want = ((unsigned long long)(J * 64 + g + SG)) << 32;
        if (!warp_spin([&] {
              return (*(volatile const unsigned long long *)&slot[g + SG - 1] &
                      0xFFFFFFFF00000000ull) == want;
            }, a.err)) {
          gave_up = true;
          break;
        }
        pz y[SG];
        bool yb = true;
#pragma unroll
        for (int v = 0; v < SG; ++v) {
          y[v] = pz_decode((uint32_t)*(volatile const unsigned long long *)&slot[g + v]);
          yb &= pz_band(y[v], 40);
          const int t = BW ? PB - 1 - (g + v) : g + v;
          if (k == 1 && lane == t) xcur = y[v];
        }
        if (!has) continue;
        if (clean && yb) {
          pz p[SG];
#pragma unroll
          for (int v = 0; v < SG; ++v) {
            const int t = BW ? PB - 1 - (g + v) : g + v;
            uint32_t sg, X0, jam;
            int S;
            pz_mul_parts(decode_band(T[t * PB + lane]), y[v], sg, S, X0, jam);
            p[v] = round_band(sg, S, X0 | jam);
          }
#pragma unroll
          for (int v = 0; v < SG; ++v) {
            uint32_t sg, X;
            int S;
            pz_add_exact_inband(xn, pz{p[v].s, p[v].m ^ 0x80000000u}, sg, S, X);
            xn = round_band(sg, S, X);
          }
        } else {
          clean = false;
#pragma unroll
          for (int v = 0; v < SG; ++v) {
            const int t = BW ? PB - 1 - (g + v) : g + v;
            xn = msub(xn, T[t * PB + lane], y[v]);
          }
        }
      }
      if (gave_up) break;
      if (has) {
        // the buffer of this parity last held block I - 2 (if this warp
        // handed one on): its reader must have copied it
        if (I - 2 >= k &&
            !warp_spin([&] { return *(volatile int *)&ex.taken[k] >= I - 2; }, a.err))
          break;
        ex.xh[I & 1][k][lane] = xn;
        if (lane == 0) ex.clean[I & 1][k] = clean;
        __threadfence_block();
        __syncwarp();
        if (lane == 0) *(volatile int *)&ex.hand[k] = I;
      }
      if (k == 1) {
        store_x(b, pipe_row0<BW>(J, nblk), a.n, xcur);
        warp_publish(&solved[J]);
      }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    return;
  }

  // ---------------------------------------------------- helper warps
  // Helper h brings blocks I = KS + 1 + h, KS + 1 + h + H, ... up to date
  // with tiles (I, J) for J <= I - KS - 1, in J order, two blocks at a time
  // (two independent chains per lane); partial sums stay in B's rows of I.
  // A tile whose words and unknowns are all in band, applied to clean
  // chains, runs on the in-band forms.  Bit k of `dirty` marks the helper's
  // k-th block as not clean (blocks past the 32nd are treated as not clean).
  uint32_t *ht = psmem + (size_t)wl * 2 * kTileWords;  // [2][kTileWords]
  const int H = (gridDim.x - 1) * PWARPS;
  const int h = (blockIdx.x - 1) * PWARPS + wl;
  const int I0 = KS + 1 + h;
  int Ilast = -1;
  for (int I = I0; I < nblk; I += H) Ilast = I;
  if (Ilast < 0) return;
  unsigned dirty = 0;
  for (int I = I0, kk = 0; I <= Ilast; I += H, ++kk) {
    const bool c = __all_sync(FULL, pz_band(load_x(b, pipe_row0<BW>(I, nblk), a.n), 80));
    if (!c || kk >= 32) dirty |= kk < 32 ? (1u << kk) : 0u;
  }
  auto is_clean = [&](int I) {
    const int kk = (I - I0) / H;
    return kk < 32 && !((dirty >> kk) & 1u);
  };
  for (int J = 0; J <= Ilast - KS - 1; ++J) {
    const int64_t c0 = pipe_row0<BW>(J, nblk);
    int I = I0;
    while (I < J + KS + 1) I += H;
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
        const int k1 = (I - I0) / H;
        if (!ok1 && k1 < 32) dirty |= 1u << k1;
        if (I2 >= 0 && !ok2) {
          const int k2 = (I2 - I0) / H;
          if (k2 < 32) dirty |= 1u << k2;
        }
      }
      store_x(b, r1, a.n, x1);
      if (I2 >= 0) store_x(b, r2, a.n, x2);
      __threadfence();
      __syncwarp();  // the tiles are read before the next pair restages them
      if (lane == 0) {
        if (J == I - KS - 1) st_release_flag(&ready[I], is_clean(I) ? 1 : 2);
        if (I2 >= 0 && J == I2 - KS - 1) st_release_flag(&ready[I2], is_clean(I2) ? 1 : 2);
      }
    }
  }
}

// x_i = (b_i - sum_{k>i, ascending} a(k, i) x_k) / a(i, i), i = n-1 .. 0,
// for one right-hand side per CTA (column blockIdx.x of B).  a(k, i) is
// A[k + i*lda] (column i below the diagonal).  The products of a row are
// formed in parallel (the next 256 while the current 256 are consumed),
// stored negated in the signed chain form with a bit per product that is NaR
// or outside the chain band; one thread runs the chain of rounded additions,
// the only serial part, in runs of PZS_RUN links by pzs_link, and takes
// pzs_link_general for a run whose start value or products are outside the
// band or whose sums cancelled two or more bits (a NaR product or b_i makes
// x_i NaR on that path).
constexpr size_t kDotStatic = 2 * ST * sizeof(pzs) + 2 * (ST / 32) * sizeof(unsigned) +
                              256 * sizeof(pzs_rtab);

__global__ void __launch_bounds__(ST, 1) trsv_dot_backward_kernel(const uint32_t *__restrict__ A,
                                                                int64_t lda, uint32_t *B,
                                                                int64_t ldb, int64_t n, int unit,
                                                                const int32_t *abort_flag) {
  static_assert(ST == 256 && PZS_RUN == 32, "one table entry per thread; a run per bad-bit word");
  __shared__ pzs prod[2][ST];
  __shared__ unsigned bad[2][ST / 32];  // bit q of word w: product 32 w + q is NaR or out of band
  __shared__ pzs_rtab tab[256];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pz *x = reinterpret_cast<pz *>(smem_raw);  // [n] the right-hand side / solution
  uint32_t *b = B + (int64_t)blockIdx.x * ldb;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (abort_flag && *abort_flag != 0) return;
  tab[tid] = pzs_rtab_entry(tid);
  for (int64_t i = tid; i < n; i += ST) x[i] = pz_decode(b[i]);
  __syncthreads();
  for (int64_t i = n - 1; i >= 0; --i) {
    const uint32_t *col = A + i * lda;
    // the negated products -a(k, i) x_k for k in [k0, k0 + ST) (zero past n)
    auto produce = [&](int64_t k0, int buf) {
      const int64_t k = k0 + tid;
      pzs p{PZS_ZERO_S, 0};
      if (k < n) {
        const pz q = pz_mul(pz_decode(col[k]), x[k]);
        p = pzs_of(pz{q.s, q.m ^ 0x80000000u});
      }
      prod[buf][tid] = p;
      const unsigned m = __ballot_sync(0xFFFFFFFFu, !pzs_in_band(p));
      if (lane == 0) bad[buf][warp] = m;
    };
    if (i + 1 < n) produce(i + 1, 0);
    __syncthreads();
    pzs acc = pzs_of(x[i]);
    int buf = 0;
    for (int64_t k0 = i + 1; k0 < n; k0 += ST) {
      if (k0 + ST < n) produce(k0 + ST, buf ^ 1);
      if (tid == 0) {
        const pzs *pr = prod[buf];
        const unsigned *bw = bad[buf];
        const int runs = (int)((min64(ST, n - k0) + PZS_RUN - 1) / PZS_RUN);
        for (int r = 0; r < runs; ++r)
          pzs_run<PZS_RUN>(acc, pr + PZS_RUN * r, PZS_RUN, tab, bw[r] == 0u);
      }
      __syncthreads();
      buf ^= 1;
    }
    if (tid == 0) {
      pz v = pz_of(acc);
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

// Shared memory a solve kernel may take per CTA: the device's opt-in limit,
// or less when the environment variable POSIT_SOLVE_SMEM_LIMIT (bytes) says
// so (room for concurrent kernels; it also makes the global-memory kernels
// for long columns run at small n).
size_t solve_smem_cap(const Limits &l) {
  size_t cap = (size_t)l.smem_optin;
  if (const char *e = getenv("POSIT_SOLVE_SMEM_LIMIT")) {
    const long long v = atoll(e);
    if (v >= 0 && (unsigned long long)v < cap) cap = (size_t)v;
  }
  return cap;
}

int laswp_vec(uint32_t *B, int64_t ldb, int64_t n, int64_t nrhs, const int32_t *ipiv,
              bool reverse, const Limits &l, cudaStream_t stream) {
  size_t smem = (size_t)n * 4;
  if (smem + 1024 <= solve_smem_cap(l)) {
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
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPipeLaunchSmem) !=
      cudaSuccess)
    return POSIT_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PT, kPipeLaunchSmem) != cudaSuccess ||
      per_sm < 1)
    return POSIT_ERR_CUDA;
  const int64_t resident = (int64_t)per_sm * l.sms;
  // One block per helper warp keeps the helpers well ahead of the pipeline;
  // down to about two blocks per helper they still keep up (two chains per
  // lane), so fewer helpers are used when that lets every right-hand side of
  // the chunk run in one launch.  With fewer co-resident warps than that
  // each helper takes more blocks (slower, still correct).  The first CTA
  // holds the diagonal and streaming warps; helpers exist when some block
  // lies beyond the streaming warps' reach.
  int64_t chunk = min64(min64(NRHS_CHUNK, nrhs),
                        (int64_t)((scratch_bytes - kPipeHead) / per_rhs));
  chunk = max64(1, chunk);
  const int64_t helpers = max64(0, nblk - KS - 1);
  const int64_t gx_full = 1 + ceil_div(helpers, PWARPS);
  const int64_t gx_min = 1 + ceil_div(ceil_div(helpers, 2), PWARPS);
  const int64_t gx = min64(max64(gx_min, min64(gx_full, resident / chunk)), resident);
  if (helpers > 0 && gx < 2) return POSIT_ERR_DEVICE;  // the helpers need a CTA of their own
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
                                    kPipeLaunchSmem, stream) != cudaSuccess)
      return POSIT_ERR_CUDA;
  }
  return POSIT_OK;
}

int trsv_dot_backward(const uint32_t *A, int64_t lda, int unit, uint32_t *B, int64_t ldb,
                      int64_t n, int64_t nrhs, const Limits &l, cudaStream_t stream,
                      const int32_t *abort_flag = nullptr) {
  size_t smem = (size_t)n * sizeof(pz);
  if (smem + kDotStatic + 1024 <= solve_smem_cap(l)) {
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
