// Tensor-core (tcgen05) kernels of the fragment ERIs, Eq. 19:
//     E = sum_q B^q B^q^H   with  B^q = M^q L^q   (V^q = L^q L^q^H).
// syrk_tc_kernel forms E (below); mlgemm_tc_kernel forms B (further down, with
// four slices instead of three).
//
// Structural zeros of L^q.  Pi^q is factorised with truncation to rank r_q
// (pivots perm_q[0..r_q)), W = L_S^{-1} is nonzero only in the columns
// perm_q[c], and V_xi = L_xi L_xi^H has rank n_q <= r_q, so L^q = W^T L_xi is
// nonzero only in the rows perm_q[c], c < r_q, and the columns J < n_q.
// B^q = M^q L^q therefore contracts over the r_q gathered columns of M^q and
// has n_J = max_q n_q columns; nothing else of L^q is touched.
//
// E as a real symmetric matrix.  The AO basis is real and the k-mesh
// Gamma-centred, so V^{-q} = conj(V^q) and M^{-q}_{(qp)} = conj(M^q_{(pq)}), hence
// E_{s(a) s(b)} = conj(E_ab) with s((pq)) = (qp).  That antiunitary symmetry fixes
// the basis  u_(pq) = e_(pq) + e_(qp),  v_(pq) = i (e_(pq) - e_(qp))  (p < q)  and
// e_(pp), so E is real in it.  The pair products are formed in that basis
// (rows u: 2 Re(conj(t_p) t_q), v: 2 Im(conj(t_p) t_q), pp: |t_p|^2, all real), so
// the rows R^q of M^q and B^q = M^q L^q are already those of the basis, with
// M^{-q} = conj(M^q); E' = sum_{all q} R^q R^q^H is real, i.e.
//     E' = c sum_{q in S} [Re R^q, Im R^q] [Re R^q, Im R^q]^T
// (c = 2 over the half set S of the time-reversal pairing, c = 1 over every q).
// One real SYRK of n_f^2 rows replaces the complex HERK: half its real
// products.  Only lower-triangle tiles are formed; the finish maps E' to E.
//
// Precision.  Each real row of R is scaled by a power of two 2^e so that its
// largest entry lies in [64, 128), and every scaled value x is written as two
// fp16 slices
//     x = s1 + s2 + d,   s1 = rint(x) (an integer, |s1| <= 128),  s2 = fp16(x - s1) (|s2| <= 1/2),
// so that |d| <= 2^-12 |s2| (19 significant bits, against 24 in FP32).  The
// tcgen05.mma kind::f16 products feed two FP32 TMEM accumulators:
//     g0 = S1.T1   (integers of magnitude <= 2^14),
//     g1 = S1.T2 + S2.T1 + S2.T2   (magnitude <= 2^6 + 2^-2 per product).
// g0 carries the bulk of E' and must be exact: a chunk of 1024 k-steps keeps
// its partial sums integers of magnitude at most 2^24, so the FP32
// accumulation is exact whatever its rounding.  g1 is not exact, but its
// products are 2^-7 of g0's and of either sign (s2 is a rounding remainder),
// so the truncation of tcgen05's FP32 accumulation over two chunks enters at
// ~2^-30 of |R_a||R_b|.  Both accumulators are double-buffered, g0 drained every
// chunk and g1 every second chunk (overlapping the next chunk's MMAs), into
// float-float (TwoSum) running sums held in the drain warps' registers.  Four products per useful
// product (the three-slice form with the same accuracy target needs six); the
// representation error d is random in sign off the diagonal, and the slicing
// kernel sums each row's sum of x^2 - (s1 + s2)^2 in FP64 so that the finish
// makes the diagonal exact.  Simulated on the c2 and c4 k-mesh data against the
// exact FP64 products: ERIs within ~1e-9 Ha, E_J within ~3e-8 Ha.
//
// Kernel roles (576 threads): warp 0 issues TMA loads, warp 1 allocates TMEM
// and issues the MMAs, warps 2-17 drain TMEM into the float-float sums.
// Every wait is bounded: on expiry the CTA records an error code and exits.
#include <cuda.h>
#include <cuda_fp16.h>

#include <cstring>
#include <vector>

#include <algorithm>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace isdf {

namespace tc {

constexpr int BM = 128;        // A' rows per tile (64 complex rows of E)
constexpr int BN = 128;        // B' rows per tile (complex columns of E)
constexpr int BK = 64;         // fp16 per row per stage (one 128-byte swizzle row)
constexpr int STAGES = 2;                   // B = M L pipeline depth
constexpr int NSLICE = 2;                   // fp16 slices per value in E': s1 (integer), s2 (remainder)
constexpr int TMEM_COLS = 512;              // g0 and g1, each two 128-column FP32 buffers
constexpr int NTHREADS = 192;
// E' kernel: warp 0 TMA, warp 1 MMA, 16 drain warps (TMEM lane quarter warp % 4, 32 of
// the 128 columns each), whose registers hold the tile's float-float running sums
constexpr int kSyrkThreads = 576, kDrainWarps = 16, kDrainCols = 32;
constexpr int kP1 = 2;                      // chunks per g1 drain
// Instruction descriptor of kind::f16: FP32 accumulate, fp16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

struct TileArgs {
  const int2* tiles;   // (ti, tj) per CTA
  float* ws_hi;        // [tile][BN][BM] float-float sums, high part
  float* ws_lo;        // low part
  int nkb;             // k-blocks of BK
  int accumulate;      // 1: add to the workspace of an earlier launch (K chunks)
  int* err;            // device error word
};

// Pipeline variants: BKt fp16 of K per stage row (64: 128-byte swizzle, 32: 64-byte
// swizzle) and NST stages; a 1024-element exact chunk of g0 is 1024 / BKt k-blocks.
// TMEM columns: g0 of chunk c at (c & 1) BN, g1 of chunk c at (2 + (c / kP1 & 1)) BN.
template <int BKt, int NST>
__global__ void __launch_bounds__(kSyrkThreads, 1)
    syrk_tc_kernel(const __grid_constant__ CUtensorMap mS1, const __grid_constant__ CUtensorMap mS2, TileArgs args) {
  constexpr int kA = BM * BKt * 2, kB = BN * BKt * 2, kStage = NSLICE * (kA + kB);
  constexpr int kChunk = 1024 / BKt;  // k-blocks per exact g0 chunk
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment of the shared-window address (swizzle atoms)
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NST * kStage);
  uint64_t* full = bars;                // [NST]
  uint64_t* empty = bars + NST;         // [NST]
  uint64_t* accf = bars + 2 * NST;      // [2] chunk accumulated (per buffer pair)
  uint64_t* acce = bars + 2 * NST + 2;  // [2] g0 buffer drained
  uint64_t* acce1 = bars + 2 * NST + 4; // [2] g1 buffer drained
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 2 * NST + 6);
  volatile int* s_err = reinterpret_cast<volatile int*>(s_tmem + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int2 tile = args.tiles[blockIdx.x];
  const int nkb = args.nkb;
  const int nchunks = (nkb + kChunk - 1) / kChunk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], kDrainWarps);
      mbar_init(&acce1[b], kDrainWarps);
    }
    *s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      // stage layout: S1 rows of A, S2 rows of A, S1 rows of B, S2 rows of B
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % NST, r = kb / NST;
        if (!mbar_wait(&empty[s], (r & 1) ^ 1, s_err, args.err, 1)) break;
        uint8_t* st = smem + s * kStage;
        mbar_expect_tx(&full[s], kStage);
        const int x = kb * BKt;
        tma_load_2d(st, &mS1, &full[s], x, tile.x * BM);
        tma_load_2d(st + kA, &mS2, &full[s], x, tile.x * BM);
        tma_load_2d(st + 2 * kA, &mS1, &full[s], x, tile.y * BN);
        tma_load_2d(st + 2 * kA + kB, &mS2, &full[s], x, tile.y * BN);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % NST, r = kb / NST;
        const int c = kb / kChunk;
        const bool first_in_chunk = (kb % kChunk) == 0;
        const int p = c / kP1;  // g1 period
        const bool first_in_period = first_in_chunk && (c % kP1) == 0;
        if (first_in_chunk) {
          // g0 buffer (c & 1) was last used by chunk c - 2, g1 buffer (p & 1) by period p - 2
          if (c >= 2 && !mbar_wait(&acce[c & 1], ((c >> 1) - 1) & 1, s_err, args.err, 2)) break;
          if (first_in_period && p >= 2 && !mbar_wait(&acce1[p & 1], ((p >> 1) - 1) & 1, s_err, args.err, 5))
            break;
          tc_fence_after();
        }
        if (!mbar_wait(&full[s], r & 1, s_err, args.err, 3)) break;
        tc_fence_after();
        const uint8_t* st = smem + s * kStage;
        const uint64_t a1 = sdesc_k<BKt>(st), a2 = sdesc_k<BKt>(st + kA);
        const uint64_t b1 = sdesc_k<BKt>(st + 2 * kA), b2 = sdesc_k<BKt>(st + 2 * kA + kB);
        const uint32_t g0 = tmem_base + (uint32_t)((c & 1) * BN), g1 = tmem_base + (uint32_t)((2 + (p & 1)) * BN);
#pragma unroll
        for (int kk = 0; kk < BKt / 16; ++kk) {
          const uint64_t off = (uint64_t)(kk * 32) >> 4;  // 16 fp16 = 32 bytes along K
          const uint32_t acc0 = (first_in_chunk && kk == 0) ? 0u : 1u;
          const uint32_t acc1 = (first_in_period && kk == 0) ? 0u : 1u;
          umma_f16(g0, a1 + off, b1 + off, kIdesc, acc0);
          umma_f16(g1, a1 + off, b2 + off, kIdesc, acc1);
          umma_f16(g1, a2 + off, b1 + off, kIdesc, 1u);
          umma_f16(g1, a2 + off, b2 + off, kIdesc, 1u);
        }
        umma_commit(&empty[s]);
        if ((kb % kChunk) == kChunk - 1 || kb == nkb - 1) umma_commit(&accf[c & 1]);
      }
    }
  } else {
    // drain warps 2..17: TMEM lane quarter warp % 4 (a hardware rule), 32 columns each;
    // the tile's float-float sums stay in registers until the last chunk
    const int q = warp & 3, cblk = (warp - 2) >> 2;
    const int row = q * 32 + lane, col0 = cblk * kDrainCols;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    float* __restrict__ wh = args.ws_hi + (size_t)blockIdx.x * BN * BM;
    float* __restrict__ wl = args.ws_lo + (size_t)blockIdx.x * BN * BM;
    float H[kDrainCols], L[kDrainCols];
#pragma unroll
    for (int j = 0; j < kDrainCols; ++j) {
      H[j] = args.accumulate ? wh[(size_t)(col0 + j) * BM + row] : 0.f;
      L[j] = args.accumulate ? wl[(size_t)(col0 + j) * BM + row] : 0.f;
    }
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      ok = __all_sync(0xffffffffu, mbar_wait(&accf[c & 1], (c >> 1) & 1, s_err, args.err, 4));
      if (!ok) break;
      tc_fence_after();
      const int p = c / kP1;
      const bool drain1 = (c % kP1) == kP1 - 1 || c == nchunks - 1;
      const uint32_t t0 = tmem_base + lane_off + (uint32_t)((c & 1) * BN + col0);
      const uint32_t t1 = tmem_base + lane_off + (uint32_t)((2 + (p & 1)) * BN + col0);
#pragma unroll
      for (int cb = 0; cb < kDrainCols / 4; ++cb) {
        uint32_t v0[4], v1[4];
        tmem_ld4(t0 + cb * 4, v0);
        if (drain1) tmem_ld4(t1 + cb * 4, v1);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int jj = cb * 4 + j;
          const float a0 = __uint_as_float(v0[j]);
          // (H, L) += a0 with TwoSum on the high part; g1 into the low part
          const float S = H[jj] + a0;
          const float bp = S - H[jj];
          const float e = (H[jj] - (S - bp)) + (a0 - bp);
          H[jj] = S;
          float l = L[jj] + e;
          if (drain1) l += __uint_as_float(v1[j]);
          L[jj] = l;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&acce[c & 1]);
        if (drain1) mbar_arrive(&acce1[p & 1]);
      }
    }
    if (ok) {
#pragma unroll
      for (int j = 0; j < kDrainCols; ++j) {
        wh[(size_t)(col0 + j) * BM + row] = H[j];
        wl[(size_t)(col0 + j) * BM + row] = L[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                 : "memory");
  }
}

// ----------------------------------------------------------------- helpers
// B is addressed as element (a, k), k = Q nJ + J, at B[slot(Q) sQ + a sA + J]
// (J < nJ), slot(Q) = qmap[Q], or Q without a map.
struct BView {
  const float2* p;
  int64_t sQ, sA, nJ;
  const int* qmap;
  __device__ __forceinline__ float2 at(int64_t a, int64_t k) const {
    const int64_t Q = k / nJ, J = k - Q * nJ;
    const int64_t slot = qmap ? (int64_t)__ldg(qmap + Q) : Q;
    return p[slot * sQ + a * sA + J];
  }
};

__device__ __forceinline__ float amax2(float2 v) { return fmaxf(fabsf(v.x), fabsf(v.y)); }
// Exponent e with m 2^e in [64, 128) (0 for a zero or non-finite maximum).
__device__ __forceinline__ int slice_exp(float m) { return (m > 0.f && isfinite(m)) ? 6 - ilogbf(m) : 0; }

template <typename T>
__device__ __forceinline__ T block_max(T v, T* sm) {
  for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  T m = sm[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = max(m, sm[i]);
  __syncthreads();
  return m;
}

// Row exponents of R over the whole sum (one block per row).  The rows of B^q
// are those of the time-reversal basis: pair o = (p < q) -> rows 2o (u) and
// 2o + 1 (v), diagonal p -> row 2P + p; R^q = [Re B^q, Im B^q].
__global__ void rrow_scale_kernel(BView B, int64_t K, int* __restrict__ row_exp) {
  const int64_t a = blockIdx.x;
  float m = 0.f;
  for (int64_t k = threadIdx.x; k < K; k += blockDim.x) m = fmaxf(m, amax2(B.at(a, k)));
  __shared__ float sm[32];
  m = block_max(m, sm);
  if (threadIdx.x == 0) row_exp[a] = slice_exp(m);
}

// Two slices of x = v 2^ex (|x| < 128): the integer s1 = rint(x) and the fp16
// remainder s2 = fp16(x - s1); dd = x - s1 - s2 exactly (FP32).
__device__ __forceinline__ void slice2(float v, int ex, float& s1, __half& s2, float& dd) {
  const float x = ldexpf(v, ex);
  s1 = rintf(x);
  const float r = x - s1;
  s2 = __float2half_rn(r);
  dd = r - __half2float(s2);
}

// Slices of the R rows for the sum positions j0 .. j0 + nq - 1, one block per
// row a: columns 2 (jl nJ + J) and + 1 hold the (re, im) of B at (position
// j0 + jl, J); columns beyond 2 nq nJ (up to the padded width K2) are zero.
// With corr, the block also adds to corr[a] the part of E'_aa (in slice units)
// that the slices do not represent, sum of x^2 - (s1 + s2)^2 = dd (2 x - dd), so
// that the finish makes the diagonal exact; off the diagonal the representation
// error is of either sign and averages out.
__global__ void __launch_bounds__(256) rsplit_kernel(BView B, int64_t j0, int nq, int64_t K2,
                                                     const int* __restrict__ row_exp, __half* __restrict__ S1,
                                                     __half* __restrict__ S2, double* __restrict__ corr) {
  const int64_t a = blockIdx.x, half = K2 / 2, ncol = (int64_t)nq * B.nJ;
  const int ex = row_exp[a];
  float d = 0.f;
  for (int64_t c2 = threadIdx.x; c2 < half; c2 += blockDim.x) {
    const float2 x = (c2 < ncol) ? B.at(a, j0 * B.nJ + c2) : make_float2(0.f, 0.f);
    float r1, i1, rd, id;
    __half r2, i2;
    slice2(x.x, ex, r1, r2, rd);
    slice2(x.y, ex, i1, i2, id);
    const int64_t at = a * K2 + 2 * c2;
    *reinterpret_cast<__half2*>(S1 + at) = __floats2half2_rn(r1, i1);
    *reinterpret_cast<__half2*>(S2 + at) = __halves2half2(r2, i2);
    d += rd * (2.f * ldexpf(x.x, ex) - rd) + id * (2.f * ldexpf(x.y, ex) - id);
  }
  if (!corr) return;
  __shared__ double sd[8];
  double v = d;
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sd[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sd[w];
    corr[a] += t;
  }
}

// The E' -> E map fused with the chemist's permutation and the traces, so that E
// is never stored.  Orbit o1 (a pair p < q: rows u = 2 o1, v = 2 o1 + 1; or a
// diagonal p: one row) and orbit o2 (x < y or x) span a block of E':
// U = E'(u1, u2), X = E'(u1, v2), Y = E'(v1, u2), Z = E'(v1, v2).  Its ERIs are
//   pair-pair:  (pq|yx) = [(U+Z) + i(Y-X)]/4,  (pq|xy) = [(U-Z) + i(X+Y)]/4,
//               (qp|yx) = conj (pq|xy),       (qp|xy) = conj (pq|yx);
//   pair-diag:  (pq|xx) = (U + iY)/2,  (qp|xx) = conj;
//   diag-pair:  (pp|yx) = (U - iX)/2,  (pp|xy) = conj;     diag-diag: (pp|xx) = U.
// For a Hermitian gamma the four terms of a block in E_J = 1/2 sum gamma_pq gamma_rs (pq|rs)
// and E_K = -1/4 sum gamma_ps gamma_rq (pq|rs) pair up into real parts:
//   J_block = U Re A Re B - Z Im A Im B + X Re A Im B - Y Im A Re B   (A = gamma_pq, B = gamma_yx),
//   K_block = 2 Re(gamma_px gamma_yq (pq|yx)) + 2 Re(gamma_py gamma_xq (pq|xy)),
// and the pair-diagonal and diagonal cases likewise, so the traces take a few
// real FP64 operations per block instead of complex ones per ERI.  Each thread
// takes one block with o1 >= o2 (consecutive threads: consecutive o1, so the
// workspace reads of the lower triangle are contiguous) and its mirror (o2, o1),
// whose values are (U, Y, X, Z).  Values are formed in float-float, the ERIs
// written as complex64 (mixed) or complex128 (FP64_TC); eri may be NULL, and
// gamma NULL skips the traces.  Per-block partials go to part[blk] (J) and
// part[gridDim.x + blk] (K); the fixed grid keeps the sums reproducible.
__device__ __forceinline__ ffloat ep_ff(const float* __restrict__ wh, const float* __restrict__ wl,
                                        const int* __restrict__ tile_of, int nt, int64_t i, int64_t j,
                                        const int* __restrict__ row_exp, ffloat sc) {
  if (i < j) {
    const int64_t t = i;
    i = j;
    j = t;
  }
  const int t = tile_of[(i / BM) * nt + (j / BN)];
  const size_t base = ((size_t)t * BN + (size_t)(j % BN)) * BM + (size_t)(i % BM);
  const ffloat v = ff_two_sum(wh[base], wl[base]);
  return ff_ldexp(v, -(row_exp[i] + row_exp[j])) * sc;
}

__device__ __forceinline__ void put_c(float2* e, double re, double im) { *e = make_float2((float)re, (float)im); }
__device__ __forceinline__ void put_c(double2* e, double re, double im) { *e = make_double2(re, im); }

struct BlockVals {
  double U, X, Y, Z;
};

// ERIs and trace terms of the block (row orbit (p, q), column orbit (x, y)); a
// diagonal orbit has q == p (resp. y == x).
template <typename TO>
__device__ __forceinline__ void emit_block(TO* __restrict__ eri, const double2* __restrict__ g, int nf, int p,
                                           int q, int x, int y, const BlockVals& b, double& aj, double& ak) {
  const bool pr = p != q, pc = x != y;
  auto at = [&](int i0, int i1, int i2, int i3) { return eri + (((int64_t)i0 * nf + i1) * nf + i2) * nf + i3; };
  auto gm = [&](int i, int j) { return g[(int64_t)i * nf + j]; };
  if (pr && pc) {
    const double r1 = 0.25 * (b.U + b.Z), i1 = 0.25 * (b.Y - b.X), r2 = 0.25 * (b.U - b.Z), i2 = 0.25 * (b.X + b.Y);
    if (eri) {
      put_c(at(p, q, y, x), r1, i1);
      put_c(at(p, q, x, y), r2, i2);
      put_c(at(q, p, y, x), r2, -i2);
      put_c(at(q, p, x, y), r1, -i1);
    }
    if (g) {
      const double2 A = gm(p, q), B = gm(y, x);
      aj += b.U * A.x * B.x - b.Z * A.y * B.y + b.X * A.x * B.y - b.Y * A.y * B.x;
      const double2 w1 = cmul(gm(p, x), gm(y, q)), w2 = cmul(gm(p, y), gm(x, q));
      ak += 2.0 * (w1.x * r1 - w1.y * i1 + w2.x * r2 - w2.y * i2);
    }
  } else if (pr) {
    const double r = 0.5 * b.U, im = 0.5 * b.Y;
    if (eri) {
      put_c(at(p, q, x, x), r, im);
      put_c(at(q, p, x, x), r, -im);
    }
    if (g) {
      const double2 A = gm(p, q);
      aj += gm(x, x).x * (A.x * b.U - A.y * b.Y);
      const double2 w = cmul(gm(p, x), gm(x, q));
      ak += 2.0 * (w.x * r - w.y * im);
    }
  } else if (pc) {
    const double r = 0.5 * b.U, im = -0.5 * b.X;
    if (eri) {
      put_c(at(p, p, y, x), r, im);
      put_c(at(p, p, x, y), r, -im);
    }
    if (g) {
      const double2 B = gm(y, x);
      aj += gm(p, p).x * (B.x * b.U + B.y * b.X);
      const double2 w = cmul(gm(p, x), gm(y, p));
      ak += 2.0 * (w.x * r - w.y * im);
    }
  } else {
    if (eri) put_c(at(p, p, x, x), b.U, 0.0);
    if (g) {
      const double2 w = gm(p, x);
      aj += gm(p, p).x * gm(x, x).x * b.U;
      ak += (w.x * w.x + w.y * w.y) * b.U;
    }
  }
}

template <typename TO>
__global__ void __launch_bounds__(256) syrk_eri_kernel(const float* __restrict__ wh, const float* __restrict__ wl,
                                                       const int* __restrict__ tile_of, int nt,
                                                       const int2* __restrict__ orb, int nf,
                                                       const int* __restrict__ row_exp, const double* __restrict__ corr,
                                                       double scale, TO* __restrict__ eri,
                                                       const double2* __restrict__ gam, double2* __restrict__ part) {
  const int no = nf * (nf + 1) / 2, P = nf * (nf - 1) / 2;
  const int nch = (no + 255) / 256;
  const int64_t ntask = (int64_t)no * nch;
  const ffloat sc(scale);
  double aj = 0.0, ak = 0.0;
  for (int64_t task = blockIdx.x; task < ntask; task += gridDim.x) {
    const int o2 = (int)(task / nch), o1 = (int)(task % nch) * 256 + (int)threadIdx.x;
    if (o1 < o2 || o1 >= no) continue;
    const int2 r = orb[o1], c = orb[o2];
    const bool pr = o1 < P, pc = o2 < P;
    const int64_t u1 = pr ? 2 * (int64_t)o1 : 2 * (int64_t)P + (o1 - P);
    const int64_t u2 = pc ? 2 * (int64_t)o2 : 2 * (int64_t)P + (o2 - P);
    BlockVals b{0.0, 0.0, 0.0, 0.0};
    b.U = ep_ff(wh, wl, tile_of, nt, u1, u2, row_exp, sc).to_double();
    if (pc) b.X = ep_ff(wh, wl, tile_of, nt, u1, u2 + 1, row_exp, sc).to_double();
    if (pr) b.Y = ep_ff(wh, wl, tile_of, nt, u1 + 1, u2, row_exp, sc).to_double();
    if (pr && pc) b.Z = ep_ff(wh, wl, tile_of, nt, u1 + 1, u2 + 1, row_exp, sc).to_double();
    if (o1 == o2 && corr) {
      // the diagonal's products left out of the contraction (slice units)
      b.U += ldexp(corr[u1], -2 * row_exp[u1]) * scale;
      if (pr) b.Z += ldexp(corr[u1 + 1], -2 * row_exp[u1 + 1]) * scale;
    }
    emit_block<TO>(eri, gam, nf, r.x, r.y, c.x, c.y, b, aj, ak);
    if (o1 != o2) emit_block<TO>(eri, gam, nf, c.x, c.y, r.x, r.y, BlockVals{b.U, b.Y, b.X, b.Z}, aj, ak);
  }
  if (!gam) return;
  __shared__ double sj[256], sk[256];
  sj[threadIdx.x] = aj;
  sk[threadIdx.x] = ak;
  __syncthreads();
  for (int o = 128; o; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sj[threadIdx.x] += sj[threadIdx.x + o];
      sk[threadIdx.x] += sk[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = make_double2(sj[0], 0.0);
    part[gridDim.x + blockIdx.x] = make_double2(sk[0], 0.0);
  }
}

// out4 = (E_J, E_K, Im E_J, Im E_K) from the per-block partials (one block, fixed order).
__global__ void __launch_bounds__(256) eri_traces_final_kernel(const double2* __restrict__ part, int nblk,
                                                               double* __restrict__ out4) {
  __shared__ double2 sj[256], sk[256];
  double2 aj = make_double2(0.0, 0.0), ak = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    aj = cadd(aj, part[i]);
    ak = cadd(ak, part[nblk + i]);
  }
  sj[threadIdx.x] = aj;
  sk[threadIdx.x] = ak;
  __syncthreads();
  for (int o = 128; o; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sj[threadIdx.x] = cadd(sj[threadIdx.x], sj[threadIdx.x + o]);
      sk[threadIdx.x] = cadd(sk[threadIdx.x], sk[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out4[0] = 0.5 * sj[0].x;
    out4[1] = -0.25 * sk[0].x;
    out4[2] = 0.5 * sj[0].y;
    out4[3] = -0.25 * sk[0].y;
  }
}

// ---------------------------------------------------------------------------
// B^q = M^q L^q on the tensor cores with three slices per operand.
//
// Only the structural nonzeros of L^q enter (see the top of the file): the
// contraction runs over c < r_q with M^q's column perm_q[c] and L^q's row
// perm_q[c], and the output has n_J columns.  Real form: one A' row per row of M,
// P_a = (Re M_a,perm(c), Im M_a,perm(c))_c, and two B' rows per column of L,
// R_J = (Re L_perm(c)J, -Im L_perm(c)J)_c and I_J = (Im L_perm(c)J, Re L_perm(c)J)_c,
// so P_a.R_J = Re B_aJ and P_a.I_J = Im B_aJ (the complex embedding sits on the
// small operand; the slices of M are written and streamed once).  M rows are
// scaled by 2^e_a (largest gathered
// component over the q of the sum in [64, 128)), L columns by 2^f_qJ per q; both
// are cut into an integer and two fp16 remainders,
//     x = s1 + s2 + s3 + d,  s1 = rint(x),  s2 = fp16(x - s1),  s3 = fp16(x - s1 - s2),
// about 30 significant bits (B = M W^T L_xi carries the cancellation of the
// ill-conditioned W, so 19 bits measurably degrade the traces).  Six fp16
// products feed three groups
//   g0 = S1T1, g1 = S1T2 + S2T1, g2 = S1T3 + S2T2 + S3T1;
// with K' = 2 r <= kMlMaxK every partial sum of g0 is an integer of magnitude
// below 2^24, so its FP32 TMEM accumulation is exact; g1 and g2 are 2^-7 and
// 2^-18 of it and accumulate in FP32 over at most kMlMaxK terms.  The epilogue
// forms g0 + (g1 + g2) once and rescales.  Simulated on the c2 data against the
// exact products: E_J within ~1e-9 Ha (four 7-bit slices with ten products: ~2e-8).
// Tiles of 128 x 64 with K rows of 32 fp16 in two stages: 72 KB of shared memory and
// 256 TMEM columns per CTA, so that two CTAs share an SM and one's set-up and
// epilogue overlap the other's MMAs (each tile runs only 2 r_q / 32 k-blocks).
constexpr int MSL = 3;                                     // slices per operand
constexpr int MBN = 64;                                    // B' rows per tile (N of the MMA)
constexpr int MBJ = MBN / 2;                               // complex columns of B per tile
constexpr int MBK = 32;                                    // fp16 of K per stage row (64-byte swizzle)
constexpr int MA_BYTES = BM * MBK * 2;                     // 8 KB per slice
constexpr int MB_BYTES = MBN * MBK * 2;                    // 4 KB per slice
constexpr int MSTAGE_BYTES = MSL * (MA_BYTES + MB_BYTES);  // 36 KB
constexpr int kMlTmem = 256;                               // three 64-column groups
constexpr int kMlMaxK = 640;                               // K' bound for exact accumulation
constexpr uint32_t kIdescMl = (1u << 4) | ((uint32_t)(MBN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

struct MlArgs {
  float2* out;          // B: element (a, J) of sum position j = j0 + ql at out[j sq + a nj + J]
  const int* qmap;      // q of each sum position
  const int* row_exp;   // e_a, [n2]
  const int* col_exp;   // f_qJ, [Nk][nj_pad] indexed by q (nj_pad: complex columns, multiple of MBJ)
  int64_t sq;           // q stride of out
  int n2, nj, nj_pad, j0, nkb;
  int* err;
};

__global__ void __launch_bounds__(NTHREADS, 2)
    mlgemm_tc_kernel(const __grid_constant__ CUtensorMap mA1, const __grid_constant__ CUtensorMap mA2,
                     const __grid_constant__ CUtensorMap mA3, const __grid_constant__ CUtensorMap mB1,
                     const __grid_constant__ CUtensorMap mB2, const __grid_constant__ CUtensorMap mB3, MlArgs args) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * MSTAGE_BYTES);
  uint64_t* full = bars;               // [STAGES]
  uint64_t* empty = bars + STAGES;     // [STAGES]
  uint64_t* accf = bars + 2 * STAGES;  // accumulation finished
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  volatile int* s_err = reinterpret_cast<volatile int*>(s_tmem + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the output-column tiles of one row block are adjacent in launch order, so
  // they run together and share the row block's slices through L2
  const int ntj = args.nj_pad / MBJ;
  const int ti = blockIdx.x / ntj, tj = blockIdx.x % ntj, ql = blockIdx.y;
  const int pos = args.j0 + ql;                      // position in the sum (storage of B)
  const int slot = args.qmap ? args.qmap[pos] : pos;  // its q (slices and exponents of L)
  const int nkb = args.nkb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    *s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(kMlTmem)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      const CUtensorMap* ma[MSL] = {&mA1, &mA2, &mA3};
      const CUtensorMap* mb[MSL] = {&mB1, &mB2, &mB3};
      const int arow = ql * args.n2 + ti * BM, brow = slot * 2 * args.nj_pad + tj * MBN;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % STAGES, r = kb / STAGES;
        if (!mbar_wait(&empty[s], (r & 1) ^ 1, s_err, args.err, 11)) break;
        uint8_t* st = smem + s * MSTAGE_BYTES;
        mbar_expect_tx(&full[s], MSTAGE_BYTES);
        const int x = kb * MBK;
#pragma unroll
        for (int i = 0; i < MSL; ++i) {
          tma_load_2d(st + i * MA_BYTES, ma[i], &full[s], x, arow);
          tma_load_2d(st + MSL * MA_BYTES + i * MB_BYTES, mb[i], &full[s], x, brow);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t g0 = tmem_base, g1 = tmem_base + MBN, g2 = tmem_base + 2 * MBN;
      bool ok = true;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int s = kb % STAGES, r = kb / STAGES;
        if (!mbar_wait(&full[s], r & 1, s_err, args.err, 12)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint8_t* st = smem + s * MSTAGE_BYTES;
        uint64_t dA[MSL], dB[MSL];
#pragma unroll
        for (int i = 0; i < MSL; ++i) {
          dA[i] = sdesc_k<MBK>(st + i * MA_BYTES);
          dB[i] = sdesc_k<MBK>(st + MSL * MA_BYTES + i * MB_BYTES);
        }
#pragma unroll
        for (int kk = 0; kk < MBK / 16; ++kk) {
          const uint64_t off = (uint64_t)(kk * 32) >> 4;
          const uint32_t acc = (kb == 0 && kk == 0) ? 0u : 1u;
          umma_f16(g0, dA[0] + off, dB[0] + off, kIdescMl, acc);
          umma_f16(g1, dA[0] + off, dB[1] + off, kIdescMl, acc);
          umma_f16(g1, dA[1] + off, dB[0] + off, kIdescMl, 1u);
          umma_f16(g2, dA[0] + off, dB[2] + off, kIdescMl, acc);
          umma_f16(g2, dA[1] + off, dB[1] + off, kIdescMl, 1u);
          umma_f16(g2, dA[2] + off, dB[0] + off, kIdescMl, 1u);
        }
        umma_commit(&empty[s]);
      }
      if (ok) umma_commit(accf);
    }
  } else {
    // epilogue: warps 2..5 -> TMEM lane quarter (warp % 4); lane r is row a of M, TMEM
    // column n is B' row n of the tile: complex column Jl = n / 2, part n % 2 (Re, Im)
    const int q = warp & 3;
    const int r = q * 32 + lane;             // row of the tile
    const int64_t a = (int64_t)ti * BM + r;  // row of M (of the q-point's block)
    // warp-uniform, so that the .sync.aligned TMEM loads are taken by whole warps
    const bool okw = __all_sync(0xffffffffu, mbar_wait(accf, 0, s_err, args.err, 13));
    tc_fence_after();
    // the operand stages are idle now: stage the 128 x MBJ complex tile for coalesced stores
    constexpr int kPitch = MBN + 2;     // floats per staged row (bank-conflict padding)
    float* tileS = reinterpret_cast<float*>(smem);
    const int ea = (okw && a < args.n2) ? args.row_exp[a] : 0;
    const int* fcol = args.col_exp + (int64_t)slot * args.nj_pad + tj * MBJ;
#pragma unroll 1
    for (int cb = 0; cb < MBN / 32; ++cb) {
      uint32_t v0[32] = {}, v1[32] = {}, v2[32] = {};
      if (okw) {
        const uint32_t lo = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(cb * 32);
        tmem_ld32(lo, v0);
        tmem_ld32(lo + MBN, v1);
        tmem_ld32(lo + 2 * MBN, v2);
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float v = __uint_as_float(v0[j]) + (__uint_as_float(v1[j]) + __uint_as_float(v2[j]));
        const int n = cb * 32 + j;
        tileS[r * kPitch + n] = ldexpf(v, -(ea + fcol[n >> 1]));
      }
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (okw) {
      const int t = threadIdx.x - 64;
      float2* outq = args.out + (int64_t)pos * args.sq;
      for (int idx = t; idx < BM * MBJ; idx += 128) {
        const int ar = idx / MBJ, Jl = idx % MBJ;
        const int64_t aa = (int64_t)ti * BM + ar;
        const int J = tj * MBJ + Jl;
        if (aa < args.n2 && J < args.nj)
          outq[aa * args.nj + J] = *reinterpret_cast<const float2*>(tileS + ar * kPitch + 2 * Jl);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kMlTmem)
                 : "memory");
  }
}

__device__ __forceinline__ float round_int(float x) { return rintf(x); }
__device__ __forceinline__ double round_int(double x) { return rint(x); }

// Three slices of v (|v| < 128): the integer s1 = rint(v) and the fp16 remainders
// s2 = fp16(v - s1), s3 = fp16(v - s1 - s2).
template <typename R>
__device__ __forceinline__ void slice3r(R v, __half& h1, __half& h2, __half& h3) {
  const R s1 = round_int(v);
  const R r1 = v - s1;
  h2 = __float2half_rn((float)r1);
  const R r2 = r1 - (R)__half2float(h2);
  h1 = __float2half_rn((float)s1);
  h3 = __float2half_rn((float)r2);
}

// Row exponents of M over the gathered columns of the q-points of the sum:
// max over positions Q < nS and c < r_q of |M^{q}_{a, perm_q[c]}|, q = qmap[Q],
// with M^q stored at position Q.
__global__ void mrow_scale_kernel(const float2* __restrict__ M, int64_t sq, int np, const int* __restrict__ qmap,
                                  int nS, const int* __restrict__ perm, const int* __restrict__ rank, int rp,
                                  int* __restrict__ row_exp) {
  const int64_t a = blockIdx.x;
  float m = 0.f;
  for (int64_t k = threadIdx.x; k < (int64_t)nS * rp; k += blockDim.x) {
    const int Q = (int)(k / rp), c = (int)(k % rp);
    const int q = qmap[Q];
    if (c < rank[q]) m = fmaxf(m, amax2(M[(int64_t)Q * sq + a * np + perm[(int64_t)q * np + c]]));
  }
  __shared__ float sm[32];
  m = block_max(m, sm);
  if (threadIdx.x == 0) row_exp[a] = slice_exp(m);
}

// A' slices of M for the sum positions j0..j0+nq-1 (M^q stored by position,
// q = qmap[j]): block ql holds row a = P_a over Kp columns: the gathered columns
// perm_q[c], c < r_q, as (re, im) pairs, zero beyond.
__global__ void msplit_kernel(const float2* __restrict__ M, int64_t sq, int np, const int* __restrict__ qmap,
                              const int* __restrict__ perm, const int* __restrict__ rank, int64_t n2, int j0, int nq,
                              int Kp, const int* __restrict__ row_exp, __half* __restrict__ S1,
                              __half* __restrict__ S2, __half* __restrict__ S3) {
  const int64_t half = Kp / 2, total = (int64_t)nq * n2 * half;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ql = e / (n2 * half), rem = e % (n2 * half);
    const int64_t a = rem / half, c = rem % half;
    const int q = qmap[j0 + ql];
    float2 v = make_float2(0.f, 0.f);
    if (c < rank[q]) v = M[(int64_t)(j0 + ql) * sq + a * np + perm[(int64_t)q * np + c]];
    const int ex = row_exp[a];
    __half r1, r2, r3, i1, i2, i3;
    slice3r<float>(ldexpf(v.x, ex), r1, r2, r3);
    slice3r<float>(ldexpf(v.y, ex), i1, i2, i3);
    const int64_t at = (ql * n2 + a) * Kp + 2 * c;
    *reinterpret_cast<__half2*>(S1 + at) = __halves2half2(r1, i1);
    *reinterpret_cast<__half2*>(S2 + at) = __halves2half2(r2, i2);
    *reinterpret_cast<__half2*>(S3 + at) = __halves2half2(r3, i3);
  }
}

// B' slices of w_q^{1/2} L^q: block (row, q), row = 2 J + part, is R_J = (Re L, -Im L)
// (part 0) or I_J = (Im L, Re L) (part 1) over the gathered rows perm_q(c) of column J,
// scaled by 2^f_qJ (largest component of the column in [64, 128)); columns J >= nj,
// c >= r_q and beyond 2 r_q are zero.  Layout [q][2 nj_pad][Kp] per slice;
// exponents [q][nj_pad].
__global__ void lslice_kernel(const double2* __restrict__ L, const double* __restrict__ sw, int np,
                              const int* __restrict__ perm, const int* __restrict__ rank, int nj, int nj_pad, int Kp,
                              __half* __restrict__ S1, __half* __restrict__ S2, __half* __restrict__ S3,
                              int* __restrict__ col_exp) {
  const int q = blockIdx.y, J = blockIdx.x >> 1, part = blockIdx.x & 1;
  const double w = sw[q];
  const int r = rank[q];
  const double2* Lq = L + (int64_t)q * np * np;
  const int* pq = perm + (int64_t)q * np;
  double m = 0.0;
  if (J < nj)
    for (int c = threadIdx.x; c < r; c += blockDim.x) {
      const double2 v = Lq[(int64_t)pq[c] * np + J];
      m = fmax(m, fmax(fabs(v.x * w), fabs(v.y * w)));
    }
  __shared__ double sm[32];
  m = block_max(m, sm);
  const int ex = (m > 0.0 && isfinite(m)) ? 6 - ilogb(m) : 0;
  if (threadIdx.x == 0 && part == 0) col_exp[(int64_t)q * nj_pad + J] = ex;
  const int64_t row = ((int64_t)q * 2 * nj_pad + blockIdx.x) * Kp;
  for (int c = threadIdx.x; c < Kp / 2; c += blockDim.x) {
    double re = 0.0, im = 0.0;
    if (J < nj && c < r) {
      const double2 v = Lq[(int64_t)pq[c] * np + J];
      const double lr = ldexp(v.x * w, ex), li = ldexp(v.y * w, ex);
      re = part ? li : lr;
      im = part ? lr : -li;
    }
    __half a1, a2, a3, b1, b2, b3;
    slice3r<double>(re, a1, a2, a3);
    slice3r<double>(im, b1, b2, b3);
    *reinterpret_cast<__half2*>(S1 + row + 2 * c) = __halves2half2(a1, b1);
    *reinterpret_cast<__half2*>(S2 + row + 2 * c) = __halves2half2(a2, b2);
    *reinterpret_cast<__half2*>(S3 + row + 2 * c) = __halves2half2(a3, b3);
  }
}

inline int nblk(int64_t total) {
  int64_t nb = (total + 255) / 256;
  if (nb > 152 * 32) nb = 152 * 32;
  return nb < 1 ? 1 : (int)nb;
}

inline int64_t round_up(int64_t x, int64_t m) { return ((x + m - 1) / m) * m; }

}  // namespace tc

// ---- E = sum_q B^q B^q^H in the real symmetric form (host side)
void pair_orbits(int nf, std::vector<int2>& orb) {
  orb.clear();
  for (int p = 0; p < nf; ++p)
    for (int q = p + 1; q < nf; ++q) orb.push_back(make_int2(p, q));
  for (int p = 0; p < nf; ++p) orb.push_back(make_int2(p, p));
}

size_t syrk_tc_split_bytes(int64_t n2, int64_t kcols) {
  return (size_t)tc::NSLICE * n2 * tc::round_up(2 * kcols, tc::BK) * sizeof(__half) + 256;
}

// Lower-triangle tiles (ti >= tj) of the n2 x n2 E' in launch order, and their
// index by (ti, tj).  Every CTA streams the whole K extent of its row blocks and
// about one CTA per SM is resident, so the order decides what L2 can share:
// tiles go in bands of `band` row blocks, and within a band column by column,
// so that the ~150 CTAs of a wave read about band + 150/band row blocks instead
// of ~150.
void syrk_tc_tiles(int64_t n2, std::vector<int2>& tiles, std::vector<int>& tile_of, int band) {
  const int64_t kGroupA = band < 1 ? 1 : band;
  tiles.clear();
  const int64_t nt = (n2 + tc::BM - 1) / tc::BM;
  tile_of.assign(nt * nt, -1);
  for (int64_t t0 = 0; t0 < nt; t0 += kGroupA)
    for (int64_t tj = 0; tj < nt; ++tj)
      for (int64_t ti = t0; ti < std::min(nt, t0 + kGroupA); ++ti)
        if (ti >= tj) {
          tile_of[ti * nt + tj] = (int)tiles.size();
          tiles.push_back(make_int2((int)ti, (int)tj));
        }
}

size_t syrk_tc_ws_bytes(int64_t ntiles) { return (size_t)ntiles * tc::BN * tc::BM * 2 * sizeof(float); }

cudaError_t syrk_tc_rowscale(cudaStream_t st, const float2* B, int64_t sQ, int64_t sA, int64_t nJ, const int* qmap,
                             int nS, int64_t n2, int* row_exp) {
  tc::BView bv{B, sQ, sA, nJ, qmap};
  tc::rrow_scale_kernel<<<(unsigned)n2, 256, 0, st>>>(bv, (int64_t)nS * nJ, row_exp);
  count_launch();
  return cudaGetLastError();
}

namespace {
template <int BKt, int NST>
cudaError_t syrk_launch(cudaStream_t st, __half* const sl[tc::NSLICE], int64_t n2, int64_t K2, const int2* tiles_d,
                        int ntiles, void* ws, int accumulate, int* err) {
  using namespace tc;
  CUtensorMap m[NSLICE];
  for (int i = 0; i < NSLICE; ++i)
    if (!make_map(&m[i], sl[i], K2, n2, K2, BM, BKt)) return cudaErrorInvalidValue;
  const size_t smem = (size_t)NST * NSLICE * (BM + BN) * BKt * 2 + 1024 + 256;
  cudaError_t e = cudaFuncSetAttribute(syrk_tc_kernel<BKt, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  float* wh = reinterpret_cast<float*>(ws);
  float* wl = wh + (size_t)ntiles * BN * BM;
  TileArgs args{tiles_d, wh, wl, (int)(K2 / BKt), accumulate, err};
  syrk_tc_kernel<BKt, NST><<<ntiles, kSyrkThreads, smem, st>>>(m[0], m[1], args);
  count_launch();
  return cudaGetLastError();
}
}  // namespace

cudaError_t syrk_tc_chunk(cudaStream_t st, const float2* B, int64_t sQ, int64_t sA, int64_t nJ, const int* qmap,
                          int64_t n2, int j0, int nq, const int* row_exp, void* split, const int2* tiles_d, int ntiles,
                          void* ws, int accumulate, int* err, int cfg) {
  cudaError_t e = syrk_tc_split(st, B, sQ, sA, nJ, qmap, n2, j0, nq, row_exp, split, nullptr);
  if (e != cudaSuccess) return e;
  return syrk_tc_mma(st, split, n2, nq, nJ, tiles_d, ntiles, ws, accumulate, err, cfg);
}

cudaError_t syrk_tc_split(cudaStream_t st, const float2* B, int64_t sQ, int64_t sA, int64_t nJ, const int* qmap,
                          int64_t n2, int j0, int nq, const int* row_exp, void* split, double* corr) {
  using namespace tc;
  if (n2 <= 0 || nq <= 0) return cudaSuccess;
  if (n2 > 2147483647LL) return cudaErrorInvalidValue;
  const int64_t K2 = round_up(2 * (int64_t)nq * nJ, BK);
  __half* S1 = reinterpret_cast<__half*>(split);
  __half* S2 = S1 + (size_t)n2 * K2;
  BView bv{B, sQ, sA, nJ, qmap};
  rsplit_kernel<<<(unsigned)n2, 256, 0, st>>>(bv, j0, nq, K2, row_exp, S1, S2, corr);
  count_launch();
  return cudaGetLastError();
}

cudaError_t syrk_tc_mma(cudaStream_t st, void* split, int64_t n2, int nq, int64_t nJ, const int2* tiles_d,
                        int ntiles, void* ws, int accumulate, int* err, int cfg) {
  using namespace tc;
  if (n2 <= 0 || nq <= 0 || ntiles <= 0) return cudaSuccess;
  const int64_t K2 = round_up(2 * (int64_t)nq * nJ, BK);
  __half* S1 = reinterpret_cast<__half*>(split);
  __half* const sl[tc::NSLICE] = {S1, S1 + (size_t)n2 * K2};
  return cfg == 1 ? syrk_launch<32, 6>(st, sl, n2, K2, tiles_d, ntiles, ws, accumulate, err)
                  : syrk_launch<64, 3>(st, sl, n2, K2, tiles_d, ntiles, ws, accumulate, err);
}

constexpr int kEriBlocks = 152 * 16;  // fixed grid of the fused finish (reproducible traces)
size_t syrk_tc_eri_part_count() { return 2 * (size_t)kEriBlocks; }

template <typename TO>
static cudaError_t finish_eri_impl(cudaStream_t st, const void* ws, int ntiles, const int* tile_of_d,
                                   const int2* orb, int nf, const int* row_exp, const double* corr, double scale,
                                   TO* eri, const double2* gamma, double2* part, double* out4) {
  using namespace tc;
  if (!eri && !gamma) return cudaSuccess;
  const float* wh = reinterpret_cast<const float*>(ws);
  const float* wl = wh + (size_t)ntiles * BN * BM;
  const int64_t n2 = (int64_t)nf * nf, nt = (n2 + BM - 1) / BM;
  syrk_eri_kernel<TO><<<kEriBlocks, 256, 0, st>>>(wh, wl, tile_of_d, (int)nt, orb, nf, row_exp, corr, scale, eri,
                                                  gamma, part);
  count_launch();
  if (gamma) {
    eri_traces_final_kernel<<<1, 256, 0, st>>>(part, kEriBlocks, out4);
    count_launch();
  }
  return cudaGetLastError();
}
cudaError_t syrk_tc_finish_eri(cudaStream_t st, const void* ws, int ntiles, const int* tile_of_d, const int2* orb,
                               int nf, const int* row_exp, const double* corr, double scale, float2* eri,
                               const double2* gamma, double2* part, double* out4) {
  return finish_eri_impl<float2>(st, ws, ntiles, tile_of_d, orb, nf, row_exp, corr, scale, eri, gamma, part, out4);
}
cudaError_t syrk_tc_finish_eri_z(cudaStream_t st, const void* ws, int ntiles, const int* tile_of_d, const int2* orb,
                                 int nf, const int* row_exp, const double* corr, double scale, double2* eri,
                                 const double2* gamma, double2* part, double* out4) {
  return finish_eri_impl<double2>(st, ws, ntiles, tile_of_d, orb, nf, row_exp, corr, scale, eri, gamma, part, out4);
}

// ---- B = M L on the tensor cores, three slices (host side)
int mlgemm_tc_kp(int rp) { return (int)tc::round_up(2 * (int64_t)rp, tc::BK); }
int mlgemm_tc_nj_pad(int nj) { return (int)tc::round_up(nj, tc::MBJ); }
bool mlgemm_tc_supported(int rp) { return rp > 0 && mlgemm_tc_kp(rp) <= tc::kMlMaxK; }
size_t mlgemm_tc_lslice_bytes(int nk, int rp, int nj) {
  return (size_t)tc::MSL * nk * (2 * mlgemm_tc_nj_pad(nj)) * mlgemm_tc_kp(rp) * sizeof(__half) + 256;
}
size_t mlgemm_tc_split_bytes(int64_t n2, int rp, int nq) {
  return (size_t)tc::MSL * nq * n2 * mlgemm_tc_kp(rp) * sizeof(__half) + 256;
}

cudaError_t mlgemm_tc_prepare(cudaStream_t st, const double2* L, const double* sw, int nk, int np, const int* perm,
                              const int* rank, int rp, int nj, void* lsl, int* col_exp) {
  using namespace tc;
  const int Kp = mlgemm_tc_kp(rp), njp = mlgemm_tc_nj_pad(nj);
  const size_t per = (size_t)nk * 2 * njp * Kp;
  __half* S1 = reinterpret_cast<__half*>(lsl);
  lslice_kernel<<<dim3(2 * njp, nk), 128, 0, st>>>(L, sw, np, perm, rank, nj, njp, Kp, S1, S1 + per, S1 + 2 * per,
                                                    col_exp);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mlgemm_tc_rowscale(cudaStream_t st, const float2* M, int64_t sq, int np, const int* qmap, int nS,
                               const int* perm, const int* rank, int rp, int64_t n2, int* row_exp) {
  tc::mrow_scale_kernel<<<(unsigned)n2, 256, 0, st>>>(M, sq, np, qmap, nS, perm, rank, rp, row_exp);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mlgemm_tc_chunk(cudaStream_t st, float2* M, int64_t sq, const int* qmap, int64_t n2, int np,
                            const int* perm, const int* rank, int rp, int nj, int j0, int nq, const int* row_exp,
                            void* split, const void* lsl, const int* col_exp, int nk, int* err) {
  using namespace tc;
  if (n2 <= 0 || nq <= 0) return cudaSuccess;
  if (!mlgemm_tc_supported(rp)) return cudaErrorInvalidValue;
  const int Kp = mlgemm_tc_kp(rp), njp = mlgemm_tc_nj_pad(nj);
  const size_t pa = (size_t)nq * n2 * Kp, pb = (size_t)nk * 2 * njp * Kp;
  __half* S1 = reinterpret_cast<__half*>(split);
  msplit_kernel<<<nblk((int64_t)nq * n2 * (Kp / 2)), 256, 0, st>>>(M, sq, np, qmap, perm, rank, n2, j0, nq, Kp,
                                                                   row_exp, S1, S1 + pa, S1 + 2 * pa);
  count_launch();
  const __half* L1 = reinterpret_cast<const __half*>(lsl);
  CUtensorMap mA[MSL], mB[MSL];
  for (int i = 0; i < MSL; ++i)
    if (!make_map(&mA[i], S1 + i * pa, Kp, (int64_t)nq * n2, Kp, BM, MBK) ||
        !make_map(&mB[i], L1 + i * pb, Kp, (int64_t)nk * 2 * njp, Kp, MBN, MBK))
      return cudaErrorInvalidValue;
  const size_t smem = (size_t)STAGES * MSTAGE_BYTES + 1024 + 256;
  cudaError_t e = cudaFuncSetAttribute(mlgemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int mt = (int)((n2 + BM - 1) / BM), ntj = njp / MBJ;
  MlArgs args{M, qmap, row_exp, col_exp, sq, (int)n2, nj, njp, j0, Kp / MBK, err};
  mlgemm_tc_kernel<<<dim3(mt * ntj, nq), NTHREADS, smem, st>>>(mA[0], mA[1], mA[2], mB[0], mB[1], mB[2], args);
  count_launch();
  return cudaGetLastError();
}

}  // namespace isdf
