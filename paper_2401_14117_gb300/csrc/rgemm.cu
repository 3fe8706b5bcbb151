// rgemm.cu -- Posit(32,2) Rgemm, C = alpha op(A) op(B) + beta C
// (Sec. 3, Eq. GEMM_DEF; the paper's GPU kernels, Sec. 3.2, are four
// shared-memory-blocked kernels, one per transpose pair).
//
// Tensor cores do not apply: every product and every sum is rounded to
// Posit(32,2) in a fixed order, which is not a dense FP contraction.  The
// kernel is bound by integer instruction issue.  Per CTA:
//   * a BM x BK tile of op(A) and a BK x BN tile of op(B) are loaded from
//     global memory (coalesced along the contiguous dimension) and decoded
//     ONCE into shared memory as (scale, signed significand) pairs; the B
//     tile is pre-multiplied by alpha (t = alpha * op(B)_lj, one rounding);
//   * each thread owns a TM x TN register tile of C, kept DECODED across the
//     whole k loop, and applies c = c + t * a for l ascending -- TM*TN
//     independent dependency chains per thread, and two 16-warp CTAs per SM,
//     hide the integer pipeline latency;
//   * the scale-dependent rounding constants (half-ulp mask, kept-bits mask,
//     a power of two that brings the tie-breaking bit to bit 31, and the
//     carry fix-up constant) come from a 256-entry table in shared memory, so
//     that the tie bit and the carry are multiply-adds: the integer ALU pipe,
//     which bounds the kernel, is left the shifts, masks and selects;
//   * C is encoded to posit words once, at the end.
// The per-element order is exactly the reference-BLAS order, so the result
// does not depend on BM/BN/BK or the grid.
//
// NaR never enters the multiply-add loop: NaR absorbs every operation and
// no operation on finite posits yields NaR, so C_ij is NaR exactly when beta
// is NaR, or beta != 0 and C_ij is NaR, or (alpha != 0, k > 0 and) alpha, a
// word of row i of op(A) or of column j of op(B) is NaR.  Tiles record those
// rows and columns in shared flags while decoding (NaR words enter the
// arithmetic as 0) and the epilogue writes NaR where a flag is set.
#include "internal.cuh"

namespace posit {
namespace {

constexpr int BM = 128, BN = 64, BK = 16;
constexpr int TM = 4, TN = 4;
constexpr int NT = 512;  // (BM / TM) * (BN / TN)
constexpr int GM = BM / TM;
constexpr int64_t kGroupM = 16;  // row tiles per group of the launch order
constexpr int kOpBand = 40;       // operand scales of the in-band fast path
constexpr int kCBand = 80;        // starting C scales of the in-band fast path
static_assert((BM / TM) * (BN / TN) == NT, "thread tile");

template <int TRI>
__device__ __forceinline__ bool tri_ok(int64_t i, int64_t j) {
  return TRI == TRI_FULL || (TRI == TRI_LOWER ? i >= j : i <= j);
}

template <bool TA, bool TB, int TRI, int TMV>
__global__ void __launch_bounds__(NT, 2)
rgemm_kernel(int64_t M, int64_t N, int64_t K, uint32_t alpha,
             const uint32_t *__restrict__ A, int64_t lda,
             const uint32_t *__restrict__ B, int64_t ldb, uint32_t beta,
             uint32_t *__restrict__ C, int64_t ldc, const int32_t *__restrict__ abort_flag,
             uint32_t neg1) {
  // neg1 = 0xFFFFFFFF: the multiplier of the in-band addition's operand pick
  // (pz_add_inband_blend), an argument so that it stays a multiply-add
  constexpr int BMV = 32 * TMV;  // CTA rows: 32 row groups of TMV rows
  constexpr int GMV = BMV / TMV;
  static_assert(GMV * (BN / TN) == NT, "thread tile");
  __shared__ __align__(16) pz As[BK][BMV];
  __shared__ __align__(16) pz Bs[BK][BN];
  __shared__ int rowNaR[BMV];
  __shared__ int colNaR[BN];
  __shared__ pz_rtab rtab[256];
  __shared__ pz_rtab rtab_in[256];

  const int tid = threadIdx.x;
  const int tm = tid % GMV;  // row group: rows tm*TMV .. +TMV-1
  const int tn = tid / GMV;  // column group (one warp): cols tn*TN .. +TN-1
  // Grouped launch order (full matrices with more than kGroupM row tiles):
  // the grid is (kGroupM row tiles, column tiles, groups; the last group may
  // be partial), so consecutive CTAs take kGroupM row tiles by a run of
  // column tiles, and a wave of CTAs streams the k slices of about 2048 rows
  // of op(A) and 1200 columns of op(B), which the CTAs that share them then
  // read from L2 instead of each from DRAM.  Otherwise the grid is (row
  // tiles, column tiles, 1).
  const unsigned mt = blockIdx.z * (unsigned)kGroupM + blockIdx.x;
  if (mt >= (unsigned)((M + BMV - 1) / BMV)) return;  // the last group may be partial
  const int64_t m0 = (int64_t)mt * BMV;
  const int64_t n0 = (int64_t)blockIdx.y * BN;
  if (TRI == TRI_LOWER && n0 > m0 + BMV - 1) return;  // tile wholly above diagonal
  if (TRI == TRI_UPPER && m0 > n0 + BN - 1) return;  // tile wholly below diagonal
  if (abort_flag != nullptr && *abort_flag != 0) return;  // a factorisation failed

  const bool all_nar = beta == PZ_NAR_BITS || (alpha == PZ_NAR_BITS && K > 0);
  for (int i = tid; i < BMV; i += NT) rowNaR[i] = 0;
  for (int j = tid; j < BN; j += NT) colNaR[j] = 0;
  for (int i = tid; i < 256; i += NT) {
    rtab[i] = pz_rtab_entry(i);
    rtab_in[i] = pz_rtab_inband_entry(i);
  }

  // Accumulators: padding elements (outside C or the triangle) start at 1
  // and are never stored; they only keep the warp on the fast path.
  pz acc[TMV][TN];
  uint32_t c_nar = 0;  // bit i*TN+j: C_ij was NaR (beta != 0)
  // In-band fast path.  While every operand t = alpha op(B)_lj and op(A)_il
  // is zero or has its scale in [-40, 40], and every starting C value is zero
  // or has its scale in [-80, 80], no rounding of the accumulation sees a
  // scale outside [-108, 89], so none needs the test for the regimes of 28 or
  // more bits.  Low end: every product and sum is a multiple of 2^-107 (a
  // product has scale >= -80 and keeps at most 27 fraction bits; exact sums of
  // multiples round to multiples), so a nonzero one is at least 2^-107.  High
  // end: products are at most 2^82, and as rounding is monotone |c_k| <= B_k
  // with B_0 < 2^81, B_(k+1) = round(B_k + 2^82), which stops growing once
  // 2^82 is below half a unit in the last place: at 2^88 (f_s = 5 there),
  // whatever K is.  The flag is cleared for good by the first tile with an
  // operand outside the bounds.
  bool in_band = true;
#pragma unroll
  for (int i = 0; i < TMV; ++i) {
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int64_t r = m0 + tm * TMV + i, c = n0 + tn * TN + j;
      pz v = pz_one();
      if (r < M && c < N && tri_ok<TRI>(r, c)) {
        if (beta == 0u) {
          v = pz_zero();
        } else {
          uint32_t w = C[r + c * ldc];
          if (w == PZ_NAR_BITS) {
            c_nar |= 1u << (i * TN + j);
            v = pz_zero();
          } else {
            v = pz_decode(w);
            if (beta != PZ_ONE_BITS && !all_nar) v = pz_mul_fast(pz_decode(beta), v);
          }
        }
      }
      acc[i][j] = v;
      in_band &= pz_is_zero(v) || (v.s >= -kCBand && v.s <= kCBand);
    }
  }

  const int64_t kTot = (alpha == 0u) ? 0 : K;
  for (int64_t k0 = 0; k0 < kTot; k0 += BK) {
    __syncthreads();  // previous tile fully consumed
    bool tile_ok = in_band;
#pragma unroll
    for (int q = 0; q < (BMV * BK) / NT; ++q) {
      int e = tid + q * NT;
      int r, c;
      if (!TA) { r = e % BMV; c = e / BMV; } else { c = e % BK; r = e / BK; }
      int64_t gr = m0 + r, gk = k0 + c;
      pz v = pz_one();
      if (gr < M && gk < K) {
        uint32_t w = TA ? A[gk + gr * lda] : A[gr + gk * lda];
        if (w == PZ_NAR_BITS) {
          rowNaR[r] = 1;
          v = pz_zero();
        } else {
          v = pz_decode(w);
        }
      }
      tile_ok &= pz_is_zero(v) || (v.s >= -kOpBand && v.s <= kOpBand);
      As[c][r] = v;
    }
#pragma unroll
    for (int q = 0; q < (BK * BN) / NT; ++q) {
      int e = tid + q * NT;
      int r, c;
      if (!TB) { r = e % BK; c = e / BK; } else { c = e % BN; r = e / BN; }
      int64_t gk = k0 + r, gc = n0 + c;
      pz v = pz_one();
      if (gk < K && gc < N) {
        uint32_t w = TB ? B[gc + gk * ldb] : B[gk + gc * ldb];
        if (w == PZ_NAR_BITS) {
          colNaR[c] = 1;
          v = pz_zero();
        } else {
          v = pz_decode(w);
          // t = alpha * op(B)_lj (a NaR alpha is handled by all_nar)
          if (alpha != PZ_ONE_BITS && !all_nar) v = pz_mul_fast(pz_decode(alpha), v);
        }
      }
      tile_ok &= pz_is_zero(v) || (v.s >= -kOpBand && v.s <= kOpBand);
      Bs[r][c] = v;
    }
    in_band = __syncthreads_and(tile_ok) && in_band;

    const int kend = (int)min64(BK, K - k0);
    if (in_band) {  // uniform over the CTA
#pragma unroll 1
      for (int kk = 0; kk < kend; ++kk) {
        pz a[TMV], b[TN];
#pragma unroll
        for (int i = 0; i < TMV; ++i) a[i] = As[kk][tm * TMV + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tn * TN + j];
#pragma unroll
        for (int i = 0; i < TMV; ++i) {
#pragma unroll
          for (int j = 0; j < TN; ++j)
            acc[i][j] = pz_add_inband_blend(rtab_in, neg1, acc[i][j],
                                            pz_mul_inband(rtab_in, b[j], a[i]));
        }
      }
    } else {
#pragma unroll 1
      for (int kk = 0; kk < kend; ++kk) {
        pz a[TMV], b[TN];
#pragma unroll
        for (int i = 0; i < TMV; ++i) a[i] = As[kk][tm * TMV + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tn * TN + j];
#pragma unroll
        for (int i = 0; i < TMV; ++i) {
#pragma unroll
          for (int j = 0; j < TN; ++j)
            acc[i][j] = pz_add_tab(rtab, acc[i][j], pz_mul_tab(rtab, b[j], a[i]));
        }
      }
    }
  }

#pragma unroll
  for (int i = 0; i < TMV; ++i) {
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int64_t r = m0 + tm * TMV + i, c = n0 + tn * TN + j;
      if (r < M && c < N && tri_ok<TRI>(r, c)) {
        int lr = tm * TMV + i, lc = tn * TN + j;
        bool nar = all_nar || ((c_nar >> (i * TN + j)) & 1u) ||
                   (kTot > 0 && (rowNaR[lr] | colNaR[lc]));
        C[r + c * ldc] = nar ? PZ_NAR_BITS : pz_to_bits(acc[i][j]);
      }
    }
  }
}

template <bool TA, bool TB, int TRI>
int launch_one(dim3 grid, bool narrow, int64_t m, int64_t n, int64_t k, uint32_t alpha,
               const uint32_t *A, int64_t lda, const uint32_t *B, int64_t ldb, uint32_t beta,
               uint32_t *C, int64_t ldc, const int32_t *abort_flag, cudaStream_t stream) {
  if (narrow)
    rgemm_kernel<TA, TB, TRI, 2><<<grid, NT, 0, stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, C,
                                                           ldc, abort_flag, 0xFFFFFFFFu);
  else
    rgemm_kernel<TA, TB, TRI, TM><<<grid, NT, 0, stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, C,
                                                            ldc, abort_flag, 0xFFFFFFFFu);
  return launch_status();
}

template <int TRI>
int launch_shape(bool ta, bool tb, dim3 grid, bool narrow, int64_t m, int64_t n, int64_t k,
                 uint32_t alpha, const uint32_t *A, int64_t lda, const uint32_t *B, int64_t ldb,
                 uint32_t beta, uint32_t *C, int64_t ldc, const int32_t *abort_flag,
                 cudaStream_t stream) {
  if (!ta && !tb)
    return launch_one<false, false, TRI>(grid, narrow, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, abort_flag, stream);
  if (!ta && tb)
    return launch_one<false, true, TRI>(grid, narrow, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, abort_flag, stream);
  if (ta && !tb)
    return launch_one<true, false, TRI>(grid, narrow, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, abort_flag, stream);
  return launch_one<true, true, TRI>(grid, narrow, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, abort_flag, stream);
}

template <int TRI>
int launch_tri(bool ta, bool tb, int64_t m, int64_t n, int64_t k, uint32_t alpha,
               const uint32_t *A, int64_t lda, const uint32_t *B, int64_t ldb,
               uint32_t beta, uint32_t *C, int64_t ldc, const int32_t *abort_flag,
               cudaStream_t stream) {
  // Launches that would not fill one wave of 128 x 64 tiles (two CTAs on
  // each of the 152 SMs; e.g. the rank-32 updates of tall, narrow panels)
  // take 64 x 64 tiles instead: twice the CTAs for the same work.
  const bool narrow = ceil_div(m, BM) * ceil_div(n, BN) < 2 * 152;
  const int64_t bm = narrow ? BM / 2 : BM;
  const int64_t gx = ceil_div(m, bm);
  if (gx > 0x7FFFFFFF) return POSIT_ERR_DEVICE;
  // gridDim.y is limited to 65535: split very wide C into column chunks
  const int64_t max_cols = (int64_t)65535 * BN;
  for (int64_t c0 = 0; c0 < n; c0 += max_cols) {
    const int64_t nc = min64(max_cols, n - c0);
    const unsigned gy = (unsigned)ceil_div(nc, BN);
    const uint32_t *Bp = tb ? B + c0 : B + c0 * ldb;
    uint32_t *Cp = C + c0 * ldc;
    // a column chunk of a triangular update keeps its global diagonal: the
    // chunked path is only used for TRI_FULL (n <= 4M columns otherwise)
    const int64_t groups = ceil_div(gx, kGroupM);
    const dim3 grid = (TRI == TRI_FULL && gx > kGroupM && groups <= 65535)
                          ? dim3((unsigned)kGroupM, gy, (unsigned)groups)
                          : dim3((unsigned)gx, gy, 1);
    int st = launch_shape<TRI>(ta, tb, grid, narrow, m, nc, k, alpha, A, lda, Bp, ldb, beta, Cp,
                               ldc, abort_flag, stream);
    if (st != POSIT_OK) return st;
  }
  return POSIT_OK;
}

}  // namespace

int rgemm_launch_guarded(bool ta, bool tb, int tri, int64_t m, int64_t n, int64_t k,
                         uint32_t alpha, const uint32_t *A, int64_t lda, const uint32_t *B,
                         int64_t ldb, uint32_t beta, uint32_t *C, int64_t ldc,
                         const int32_t *abort_flag, cudaStream_t stream) {
  if (m <= 0 || n <= 0) return POSIT_OK;
  if (tri == TRI_LOWER)
    return launch_tri<TRI_LOWER>(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, abort_flag, stream);
  if (tri == TRI_UPPER)
    return launch_tri<TRI_UPPER>(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, abort_flag, stream);
  return launch_tri<TRI_FULL>(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, abort_flag, stream);
}

int rgemm_launch(bool ta, bool tb, int tri, int64_t m, int64_t n, int64_t k,
                 uint32_t alpha, const uint32_t *A, int64_t lda, const uint32_t *B,
                 int64_t ldb, uint32_t beta, uint32_t *C, int64_t ldc,
                 cudaStream_t stream) {
  return rgemm_launch_guarded(ta, tb, tri, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                              nullptr, stream);
}

}  // namespace posit

using namespace posit;

extern "C" int posit_rgemm(char transa, char transb, int64_t m, int64_t n, int64_t k,
                           posit32_t alpha, const posit32_t *A, int64_t lda,
                           const posit32_t *B, int64_t ldb, posit32_t beta,
                           posit32_t *C, int64_t ldc, cudaStream_t stream) {
  if (!valid_trans(transa)) return -1;
  if (!valid_trans(transb)) return -2;
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (k < 0) return -5;
  const bool ta = is_trans(transa), tb = is_trans(transb);
  const int64_t arows = ta ? k : m, brows = tb ? n : k;
  if (lda < max64(1, arows)) return -8;
  if (ldb < max64(1, brows)) return -10;
  if (ldc < max64(1, m)) return -13;
  if (m == 0 || n == 0) return POSIT_OK;
  if ((alpha == 0u || k == 0) && beta == PZ_ONE_BITS) return POSIT_OK;
  const bool reads_ab = alpha != 0u && k > 0;
  if (reads_ab && !A) return -7;
  if (reads_ab && !B) return -9;
  if (!C) return -12;
  return rgemm_launch(ta, tb, TRI_FULL, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream);
}
