// FP64-class tensor-core contractions of the fragment ERIs (Eq. 19), the
// ISDF_FP64_TC path:
//     B^q = M^q L^q          five exact fp16 slices per operand (mlgemm5)
//     E'  = c sum_q R^q R^qT  four exact fp16 slices per operand (syrk4)
// with M^q and B^q held in float-float (ff.cuh).  The structure is that of the
// mixed path (real symmetric form of E in the time-reversal basis, structural
// zeros of L^q); what changes is the precision of every step.
//
// Error-free slicing (Ozaki, Ogita, Oishi & Rump, 2012).  Each real row is
// scaled by 2^e so that its largest entry lies in [64, 128) and written as
//     v = s1 + s2/2^7 + s3/2^14 + ... ,  |s1| <= 128, |s_i| <= 64 (i > 1),
// each slice an integer stored exactly in fp16; the float-float value is
// renormalised (TwoSum) after each slice so that every remainder lies in
// [-1/2, 1/2].  The products of slices S_a T_b with a + b below the slice count
// feed one FP32 TMEM accumulator per weight 2^{-7(a+b)}.
//
// syrk4: groups g0..g3 (1, 2, 3, 4 products per k-step).  A chunk of 512
// k-steps keeps every partial sum of every group an integer of magnitude below
// 2^24 (g3: at most 2 (128 64) + 2 (64 64) = 1.5 2^14 per k-step), so the
// accumulation is exact; each chunk is drained into float-float sums held in
// registers: (H, L) += g0 by TwoSum, L += g1/2^7 + g2/2^14 + g3/2^21 in FP32
// (rounding ~2^-31 of |R_a||R_b|).  The dropped products and the slicing
// remainder leave ~2^-28 of |R_a||R_b|.  TMEM holds the four groups (4 x 128
// columns), so the MMAs of a chunk wait for the drain of the one before.
//
// mlgemm5: groups g0..g4 over K' = 2 r_q <= 576 (g4: at most 7 2^12 per k-step),
// exact without draining; the epilogue forms g0 + (g1/2^7 + ... + g4/2^28) as a
// float-float value (~2^-31 of |M_a||L_J|).
//
// Kernel roles: warp 0 issues TMA loads, warp 1 allocates TMEM and issues the
// MMAs, the remaining warps drain TMEM.  Every wait is bounded (tc_ptx.cuh).
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace isdf {

namespace tc64 {

using namespace tc;

constexpr int BM = 128;                  // rows per tile (A side)
constexpr int BN = 128;                  // rows per tile (B side) of E'
constexpr int BKt = 32;                  // fp16 per row and k-block (64-byte swizzle rows)
constexpr int NST = 3;                   // pipeline stages
constexpr int NS4 = 4;                   // slices of syrk4
constexpr int kA = BM * BKt * 2;         // 8 KB per slice
constexpr int kB = BN * BKt * 2;         // 8 KB per slice
constexpr int kStage4 = NS4 * (kA + kB); // 64 KB
constexpr int kChunk4 = 16;              // k-blocks per exact chunk (512 k-steps)
constexpr int NT4 = 576;                 // warp 0 TMA, warp 1 MMA, warps 2..17 drain
constexpr int kDrainCols = 32;           // columns of the running sums per drain thread
constexpr int TMEM_COLS = 512;
constexpr uint32_t kIdesc4 = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

constexpr int NS5 = 5;                   // slices of mlgemm5
constexpr int MBN = 96;                  // output columns per tile
constexpr int kMB = MBN * BKt * 2;       // 6 KB per slice
constexpr int kStage5 = NS5 * (kA + kMB);  // 70 KB
constexpr int kMl5MaxK = 576;            // K' bound of the exact accumulation
constexpr int NT5 = 192;
constexpr uint32_t kIdesc5 = (1u << 4) | ((uint32_t)(MBN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__host__ __device__ constexpr int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// NSL integer slices of the float-float value v 2^ex (largest entry of its row in [64, 128)).
template <int NSL>
__device__ __forceinline__ void slice_ff(ffloat v, int ex, __half (&out)[NSL]) {
  ffloat t = ff_two_sum(ldexpf(v.hi, ex), ldexpf(v.lo, ex));
#pragma unroll
  for (int i = 0; i < NSL; ++i) {
    const float s = rintf(t.hi);
    out[i] = __float2half_rn(s);
    // remainder (t.hi - s is exact), renormalised, times 2^7
    t = ff_two_sum(t.hi - s, t.lo);
    t.hi *= 128.f;
    t.lo *= 128.f;
  }
}

__device__ __forceinline__ float amaxff(const ffcomplex& v) { return fmaxf(fabsf(v.x.hi), fabsf(v.y.hi)); }
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


// ------------------------------------------------------------------ syrk4
struct Syrk4Args {
  const int2* tiles;  // (ti, tj) per CTA
  float* ws_hi;       // [tile][BN][BM] float-float sums (the mixed path's layout)
  float* ws_lo;
  int nkb;            // k-blocks of BKt
  int accumulate;     // 1: add to the workspace of an earlier launch
  int* err;
};

__global__ void __launch_bounds__(NT4, 1)
    syrk4_tc_kernel(const __grid_constant__ CUtensorMap m1, const __grid_constant__ CUtensorMap m2,
                    const __grid_constant__ CUtensorMap m3, const __grid_constant__ CUtensorMap m4,
                    Syrk4Args args) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NST * kStage4);
  uint64_t* full = bars;                 // [NST] stage landed
  uint64_t* empty = bars + NST;          // [NST] stage consumed by the MMAs
  uint64_t* accf = bars + 2 * NST;       // chunk accumulated
  uint64_t* drained = bars + 2 * NST + 1;  // chunk drained (one arrive per drain warp)
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 2 * NST + 2);
  volatile int* s_err = reinterpret_cast<volatile int*>(s_tmem + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int2 tile = args.tiles[blockIdx.x];
  const int nkb = args.nkb;
  const int nchunks = (nkb + kChunk4 - 1) / kChunk4;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_init(drained, (NT4 / 32) - 2);
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
      const CUtensorMap* mp[NS4] = {&m1, &m2, &m3, &m4};
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % NST, r = kb / NST;
        if (!mbar_wait(&empty[s], (r & 1) ^ 1, s_err, args.err, 21)) break;
        uint8_t* st = smem + s * kStage4;
        mbar_expect_tx(&full[s], kStage4);
        const int x = kb * BKt;
#pragma unroll
        for (int i = 0; i < NS4; ++i) {
          tma_load_2d(st + i * kA, mp[i], &full[s], x, tile.x * BM);
          tma_load_2d(st + NS4 * kA + i * kB, mp[i], &full[s], x, tile.y * BN);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t g0 = tmem_base, g1 = tmem_base + BN, g2 = tmem_base + 2 * BN, g3 = tmem_base + 3 * BN;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % NST, r = kb / NST, c = kb / kChunk4;
        const bool first = (kb % kChunk4) == 0;
        if (first && c > 0) {
          // the four groups of chunk c - 1 must have been drained
          if (!mbar_wait(drained, (c - 1) & 1, s_err, args.err, 22)) break;
          tc_fence_after();
        }
        if (!mbar_wait(&full[s], r & 1, s_err, args.err, 23)) break;
        tc_fence_after();
        const uint8_t* st = smem + s * kStage4;
        uint64_t dA[NS4], dB[NS4];
#pragma unroll
        for (int i = 0; i < NS4; ++i) {
          dA[i] = sdesc_k<BKt>(st + i * kA);
          dB[i] = sdesc_k<BKt>(st + NS4 * kA + i * kB);
        }
#pragma unroll
        for (int kk = 0; kk < BKt / 16; ++kk) {
          const uint64_t off = (uint64_t)(kk * 32) >> 4;  // 16 fp16 = 32 bytes along K
          const uint32_t a = (first && kk == 0) ? 0u : 1u;
          umma_f16(g0, dA[0] + off, dB[0] + off, kIdesc4, a);
          umma_f16(g1, dA[0] + off, dB[1] + off, kIdesc4, a);
          umma_f16(g1, dA[1] + off, dB[0] + off, kIdesc4, 1u);
          umma_f16(g2, dA[0] + off, dB[2] + off, kIdesc4, a);
          umma_f16(g2, dA[1] + off, dB[1] + off, kIdesc4, 1u);
          umma_f16(g2, dA[2] + off, dB[0] + off, kIdesc4, 1u);
          umma_f16(g3, dA[0] + off, dB[3] + off, kIdesc4, a);
          umma_f16(g3, dA[1] + off, dB[2] + off, kIdesc4, 1u);
          umma_f16(g3, dA[2] + off, dB[1] + off, kIdesc4, 1u);
          umma_f16(g3, dA[3] + off, dB[0] + off, kIdesc4, 1u);
        }
        umma_commit(&empty[s]);
        if ((kb % kChunk4) == kChunk4 - 1 || kb == nkb - 1) umma_commit(accf);
      }
    }
  } else {
    // drain warps 2..17: TMEM lane quarter warp % 4 (a hardware rule), column block (warp - 2) / 4
    const int quarter = warp & 3, cblk = (warp - 2) >> 2;
    const int row = quarter * 32 + lane, col0 = cblk * kDrainCols;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    float* __restrict__ wh = args.ws_hi + (size_t)blockIdx.x * BN * BM;
    float* __restrict__ wl = args.ws_lo + (size_t)blockIdx.x * BN * BM;
    float H[kDrainCols], L[kDrainCols];
#pragma unroll
    for (int j = 0; j < kDrainCols; ++j) {
      H[j] = 0.f;
      L[j] = 0.f;
    }
    if (args.accumulate) {
#pragma unroll
      for (int j = 0; j < kDrainCols; ++j) {
        H[j] = wh[(size_t)(col0 + j) * BM + row];
        L[j] = wl[(size_t)(col0 + j) * BM + row];
      }
    }
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      ok = __all_sync(0xffffffffu, mbar_wait(accf, c & 1, s_err, args.err, 24));
      if (!ok) break;
      tc_fence_after();
#pragma unroll
      for (int cb = 0; cb < kDrainCols / 4; ++cb) {
        // two groups at a time (register pressure: the running sums stay resident)
        uint32_t va[4], vb[4];
        float low[4];
        const uint32_t t = tmem_base + lane_off + (uint32_t)(col0 + cb * 4);
        tmem_ld4(t + 3 * BN, va);
        tmem_ld4(t + 2 * BN, vb);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 4; ++j)
          low[j] = fmaf(__uint_as_float(va[j]), 1.0f / 2097152.0f, __uint_as_float(vb[j]) * (1.0f / 16384.0f));
        tmem_ld4(t + BN, va);
        tmem_ld4(t, vb);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int jj = cb * 4 + j;
          const float a0 = __uint_as_float(vb[j]);
          const float lw = fmaf(__uint_as_float(va[j]), 1.0f / 128.0f, low[j]);
          // (H, L) += a0 with TwoSum on the high part, then the low groups
          const float S = H[jj] + a0;
          const float bp = S - H[jj];
          const float e = (H[jj] - (S - bp)) + (a0 - bp);
          H[jj] = S;
          L[jj] += e + lw;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(drained);
    }
    if (ok) {
#pragma unroll
      for (int j = 0; j < kDrainCols; ++j) {
        const ffloat v = ff_two_sum(H[j], L[j]);
        wh[(size_t)(col0 + j) * BM + row] = v.hi;
        wl[(size_t)(col0 + j) * BM + row] = v.lo;
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

// B viewed as element (a, k), k = Q nJ + J, at B[Q sQ + a sA + J] (J < nJ).
struct FFView {
  const ffcomplex* p;
  int64_t sQ, sA, nJ;
  __device__ __forceinline__ ffcomplex at(int64_t a, int64_t k) const {
    const int64_t Q = k / nJ, J = k - Q * nJ;
    return p[Q * sQ + a * sA + J];
  }
};

// Row exponents of R = [Re B, Im B] over the whole sum (one block per row).
__global__ void rrow_scale_ff_kernel(FFView B, int64_t K, int* __restrict__ row_exp) {
  const int64_t a = blockIdx.x;
  float m = 0.f;
  for (int64_t k = threadIdx.x; k < K; k += blockDim.x) m = fmaxf(m, amaxff(B.at(a, k)));
  __shared__ float sm[32];
  m = block_max(m, sm);
  if (threadIdx.x == 0) row_exp[a] = slice_exp(m);
}

// Four slices of the rows of R for the sum positions j0 .. j0 + nq - 1, one block
// per row a (columns 2 (jl nJ + J) and + 1 hold re and im; zero up to the padded
// width K2).  With corr, the block adds to corr[a] the products of the row with
// itself that the ten-product contraction leaves out (slice units):
// (2 s2 s4 + s3^2)/2^28 + 2 s3 s4/2^35 + s4^2/2^42 per value; they are of one sign
// on E'_aa only, where dropping them would bias the diagonal.
__global__ void __launch_bounds__(256) rsplit4_kernel(FFView B, int64_t j0, int nq, int64_t K2,
                                                      const int* __restrict__ row_exp, __half* __restrict__ S,
                                                      int64_t per, double* __restrict__ corr) {
  const int64_t a = blockIdx.x, half = K2 / 2, ncol = (int64_t)nq * B.nJ;
  const int ex = row_exp[a];
  double d = 0.0;
  for (int64_t c2 = threadIdx.x; c2 < half; c2 += blockDim.x) {
    ffcomplex x{ffloat(0.f, 0.f), ffloat(0.f, 0.f)};
    if (c2 < ncol) x = B.at(a, j0 * B.nJ + c2);
    __half hr[NS4], hi[NS4];
    slice_ff<NS4>(x.x, ex, hr);
    slice_ff<NS4>(x.y, ex, hi);
    const int64_t at = a * K2 + 2 * c2;
#pragma unroll
    for (int i = 0; i < NS4; ++i) *reinterpret_cast<__half2*>(S + i * per + at) = __halves2half2(hr[i], hi[i]);
    const float r2 = __half2float(hr[1]), r3 = __half2float(hr[2]), r4 = __half2float(hr[3]);
    const float i2 = __half2float(hi[1]), i3 = __half2float(hi[2]), i4 = __half2float(hi[3]);
    const float t4 = 2.f * (r2 * r4 + i2 * i4) + (r3 * r3 + i3 * i3);
    const float t5 = 2.f * (r3 * r4 + i3 * i4), t6 = r4 * r4 + i4 * i4;
    d += (double)(t4 + (t5 + t6 * (1.f / 128.f)) * (1.f / 128.f)) * (1.0 / 268435456.0);
  }
  if (!corr) return;
  __shared__ double sd[8];
  for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) sd[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sd[w];
    corr[a] += t;
  }
}

// ------------------------------------------------------------------ mlgemm5
struct Ml5Args {
  ffcomplex* out;       // B: element (a, J) of sum position j = j0 + ql at out[j sq + a nj + J]
  const int* qmap;      // q of each sum position
  const int* row_exp;   // e_a, [n2]
  const int* col_exp;   // f_qJ, [Nk][nj_pad] indexed by q
  int64_t sq;           // q stride of out
  int n2, nj, nj_pad, j0, nkb;
  int* err;
};

__global__ void __launch_bounds__(NT5, 1)
    mlgemm5_tc_kernel(const __grid_constant__ CUtensorMap a1, const __grid_constant__ CUtensorMap a2,
                      const __grid_constant__ CUtensorMap a3, const __grid_constant__ CUtensorMap a4,
                      const __grid_constant__ CUtensorMap a5, const __grid_constant__ CUtensorMap b1,
                      const __grid_constant__ CUtensorMap b2, const __grid_constant__ CUtensorMap b3,
                      const __grid_constant__ CUtensorMap b4, const __grid_constant__ CUtensorMap b5, Ml5Args args) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NST * kStage5);
  uint64_t* full = bars;               // [NST]
  uint64_t* empty = bars + NST;        // [NST]
  uint64_t* accf = bars + 2 * NST;     // accumulation finished
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 2 * NST + 1);
  volatile int* s_err = reinterpret_cast<volatile int*>(s_tmem + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntj = args.nj_pad / MBN;
  const int ti = blockIdx.x / ntj, tj = blockIdx.x % ntj, ql = blockIdx.y;
  const int pos = args.j0 + ql;                      // position in the sum (storage of B)
  const int slot = args.qmap ? args.qmap[pos] : pos;  // its q (slices and exponents of L)
  const int nkb = args.nkb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
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
      const CUtensorMap* ma[NS5] = {&a1, &a2, &a3, &a4, &a5};
      const CUtensorMap* mb[NS5] = {&b1, &b2, &b3, &b4, &b5};
      const int arow = ql * 2 * args.n2 + ti * BM, brow = slot * args.nj_pad + tj * MBN;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % NST, r = kb / NST;
        if (!mbar_wait(&empty[s], (r & 1) ^ 1, s_err, args.err, 31)) break;
        uint8_t* st = smem + s * kStage5;
        mbar_expect_tx(&full[s], kStage5);
        const int x = kb * BKt;
#pragma unroll
        for (int i = 0; i < NS5; ++i) {
          tma_load_2d(st + i * kA, ma[i], &full[s], x, arow);
          tma_load_2d(st + NS5 * kA + i * kMB, mb[i], &full[s], x, brow);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int s = kb % NST, r = kb / NST;
        if (!mbar_wait(&full[s], r & 1, s_err, args.err, 32)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint8_t* st = smem + s * kStage5;
        uint64_t dA[NS5], dB[NS5];
#pragma unroll
        for (int i = 0; i < NS5; ++i) {
          dA[i] = sdesc_k<BKt>(st + i * kA);
          dB[i] = sdesc_k<BKt>(st + NS5 * kA + i * kMB);
        }
#pragma unroll
        for (int kk = 0; kk < BKt / 16; ++kk) {
          const uint64_t off = (uint64_t)(kk * 32) >> 4;
          const uint32_t acc = (kb == 0 && kk == 0) ? 0u : 1u;
          // group g = a + b over the 15 products with a + b <= 4
#pragma unroll
          for (int g = 0; g < NS5; ++g)
#pragma unroll
            for (int a = 0; a <= g; ++a)
              umma_f16(tmem_base + (uint32_t)(g * MBN), dA[a] + off, dB[g - a] + off, kIdesc5, a == 0 ? acc : 1u);
        }
        umma_commit(&empty[s]);
      }
      if (ok) umma_commit(accf);
    }
  } else {
    // epilogue: warps 2..5 -> TMEM lane quarter (warp % 4); rows P_a / Q_a are lanes 2i / 2i+1
    const int q = warp & 3;
    const int r = q * 32 + lane;             // row of the tile
    const int64_t R = (int64_t)ti * BM + r;  // row of A'
    const int al = r >> 1, part = r & 1;
    const int64_t a = R >> 1;
    const bool okw = __all_sync(0xffffffffu, mbar_wait(accf, 0, s_err, args.err, 33));
    tc_fence_after();
    // the operand stages are idle now: stage the 64 x MBN float-float complex tile
    constexpr int kPitch = 4 * MBN + 4;  // floats per staged row
    float* tileS = reinterpret_cast<float*>(smem);
    const int ea = (okw && a < args.n2) ? args.row_exp[a] : 0;
    const int* fcol = args.col_exp + (int64_t)slot * args.nj_pad + tj * MBN;
#pragma unroll 1
    for (int cb = 0; cb < MBN / 8; ++cb) {
      uint32_t v[NS5][8];
#pragma unroll
      for (int g = 0; g < NS5; ++g)
#pragma unroll
        for (int j = 0; j < 8; ++j) v[g][j] = 0u;
      if (okw) {
        const uint32_t lo = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(cb * 8);
#pragma unroll
        for (int g = 0; g < NS5; ++g) tmem_ld8(lo + (uint32_t)(g * MBN), v[g]);
        tmem_wait_ld();
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float low =
            fmaf(__uint_as_float(v[4][j]), 1.0f / 268435456.0f,
                 fmaf(__uint_as_float(v[3][j]), 1.0f / 2097152.0f,
                      fmaf(__uint_as_float(v[2][j]), 1.0f / 16384.0f, __uint_as_float(v[1][j]) * (1.0f / 128.0f))));
        const int Jl = cb * 8 + j;
        const ffloat x = ff_ldexp(ff_two_sum(__uint_as_float(v[0][j]), low), -(ea + fcol[Jl]));
        *reinterpret_cast<float2*>(tileS + al * kPitch + 4 * Jl + 2 * part) = make_float2(x.hi, x.lo);
      }
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (okw) {
      const int t = threadIdx.x - 64;
      ffcomplex* outq = args.out + (int64_t)pos * args.sq;
      for (int idx = t; idx < (BM / 2) * MBN; idx += 128) {
        const int ar = idx / MBN, Jl = idx % MBN;
        const int64_t aa = (int64_t)ti * (BM / 2) + ar;
        const int J = tj * MBN + Jl;
        if (aa < args.n2 && J < args.nj) {
          const float4 f = *reinterpret_cast<const float4*>(tileS + ar * kPitch + 4 * Jl);
          outq[aa * args.nj + J] = ffcomplex{ffloat(f.x, f.y), ffloat(f.z, f.w)};
        }
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

// Row exponents of M over the gathered columns of the q-points of the sum (M^q
// stored at position Q, q = qmap[Q]).
__global__ void mrow_scale_ff_kernel(const ffcomplex* __restrict__ M, int64_t sq, int np, const int* __restrict__ qmap,
                                     int nS, const int* __restrict__ perm, const int* __restrict__ rank, int rp,
                                     int* __restrict__ row_exp) {
  const int64_t a = blockIdx.x;
  float m = 0.f;
  for (int64_t k = threadIdx.x; k < (int64_t)nS * rp; k += blockDim.x) {
    const int Q = (int)(k / rp), c = (int)(k % rp);
    const int q = qmap[Q];
    if (c < rank[q]) m = fmaxf(m, amaxff(M[(int64_t)Q * sq + a * np + perm[(int64_t)q * np + c]]));
  }
  __shared__ float sm[32];
  m = block_max(m, sm);
  if (threadIdx.x == 0) row_exp[a] = slice_exp(m);
}

// Five slices of the A' rows of M for the sum positions j0 .. j0 + nq - 1: row
// 2a (P_a) = (Re m, Im m) and row 2a + 1 (Q_a) = (Im m, -Re m) over the gathered
// columns perm_q[c], c < r_q, zero beyond; slice i at S + i pa.
__global__ void msplit5_kernel(const ffcomplex* __restrict__ M, int64_t sq, int np, const int* __restrict__ qmap,
                               const int* __restrict__ perm, const int* __restrict__ rank, int64_t n2, int j0, int nq,
                               int Kp, const int* __restrict__ row_exp, __half* __restrict__ S, size_t pa) {
  const int64_t half = Kp / 2, total = (int64_t)nq * n2 * half;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ql = e / (n2 * half), rem = e % (n2 * half);
    const int64_t a = rem / half, c = rem % half;
    const int q = qmap[j0 + ql];
    ffcomplex v{ffloat(0.f, 0.f), ffloat(0.f, 0.f)};
    if (c < rank[q]) v = M[(int64_t)(j0 + ql) * sq + a * np + perm[(int64_t)q * np + c]];
    const int ex = row_exp[a];
    __half hr[NS5], hi[NS5];
    slice_ff<NS5>(v.x, ex, hr);
    slice_ff<NS5>(v.y, ex, hi);
    const int64_t rP = (ql * 2 * n2 + 2 * a) * Kp + 2 * c, rQ = rP + Kp;
#pragma unroll
    for (int i = 0; i < NS5; ++i) {
      *reinterpret_cast<__half2*>(S + i * pa + rP) = __halves2half2(hr[i], hi[i]);
      *reinterpret_cast<__half2*>(S + i * pa + rQ) = __halves2half2(hi[i], __hneg(hr[i]));
    }
  }
}

// Five slices of a double value (|v| < 128).
__device__ __forceinline__ void slice_d5(double v, __half (&out)[NS5]) {
#pragma unroll
  for (int i = 0; i < NS5; ++i) {
    const double s = rint(v);
    out[i] = __float2half_rn((float)s);
    v = (v - s) * 128.0;
  }
}

// B' slices of w_q^{1/2} L^q: block (J, q) is the row (Re L_perm(c)J, -Im L_perm(c)J)_c
// scaled by 2^f_qJ (largest component in [64, 128)); zero for J >= nj, c >= r_q.
// Layout [q][nj_pad][Kp] per slice (slice i at S + i per); exponents [q][nj_pad].
__global__ void lslice5_kernel(const double2* __restrict__ L, const double* __restrict__ sw, int np,
                               const int* __restrict__ perm, const int* __restrict__ rank, int nj, int nj_pad, int Kp,
                               __half* __restrict__ S, size_t per, int* __restrict__ col_exp) {
  const int q = blockIdx.y, J = blockIdx.x;
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
  if (threadIdx.x == 0) col_exp[(int64_t)q * nj_pad + J] = ex;
  const int64_t row = ((int64_t)q * nj_pad + J) * Kp;
  for (int c = threadIdx.x; c < Kp / 2; c += blockDim.x) {
    double re = 0.0, im = 0.0;
    if (J < nj && c < r) {
      const double2 v = Lq[(int64_t)pq[c] * np + J];
      re = ldexp(v.x * w, ex);
      im = -ldexp(v.y * w, ex);
    }
    __half hr[NS5], hi[NS5];
    slice_d5(re, hr);
    slice_d5(im, hi);
#pragma unroll
    for (int i = 0; i < NS5; ++i) *reinterpret_cast<__half2*>(S + i * per + row + 2 * c) = __halves2half2(hr[i], hi[i]);
  }
}

inline int nblk(int64_t total) {
  int64_t nb = (total + 255) / 256;
  if (nb > 152 * 32) nb = 152 * 32;
  return nb < 1 ? 1 : (int)nb;
}

}  // namespace tc64

// ---- host side of the FP64-class contractions
size_t syrk4_tc_split_bytes(int64_t n2, int64_t kcols) {
  return (size_t)tc64::NS4 * n2 * tc64::rup(2 * kcols, tc64::BKt) * sizeof(__half) + 256;
}

cudaError_t syrk4_tc_rowscale(cudaStream_t st, const ffcomplex* B, int64_t sQ, int64_t sA, int64_t nJ, int nS,
                              int64_t n2, int* row_exp) {
  if (n2 <= 0) return cudaSuccess;
  tc64::rrow_scale_ff_kernel<<<(unsigned)n2, 256, 0, st>>>(tc64::FFView{B, sQ, sA, nJ}, (int64_t)nS * nJ, row_exp);
  count_launch();
  return cudaGetLastError();
}

cudaError_t syrk4_tc_split(cudaStream_t st, const ffcomplex* B, int64_t sQ, int64_t sA, int64_t nJ, int64_t n2,
                           int j0, int nq, const int* row_exp, void* split, double* corr) {
  using namespace tc64;
  if (n2 <= 0 || nq <= 0) return cudaSuccess;
  if (n2 > 2147483647LL) return cudaErrorInvalidValue;
  const int64_t K2 = rup(2 * (int64_t)nq * nJ, BKt);
  rsplit4_kernel<<<(unsigned)n2, 256, 0, st>>>(FFView{B, sQ, sA, nJ}, j0, nq, K2, row_exp,
                                              reinterpret_cast<__half*>(split), n2 * K2, corr);
  count_launch();
  return cudaGetLastError();
}

cudaError_t syrk4_tc_mma(cudaStream_t st, void* split, int64_t n2, int nq, int64_t nJ, const int2* tiles_d,
                         int ntiles, void* ws, int accumulate, int* err) {
  using namespace tc64;
  if (n2 <= 0 || nq <= 0 || ntiles <= 0) return cudaSuccess;
  const int64_t K2 = rup(2 * (int64_t)nq * nJ, BKt);
  const __half* S = reinterpret_cast<const __half*>(split);
  CUtensorMap m[NS4];
  for (int i = 0; i < NS4; ++i)
    if (!make_map(&m[i], S + (size_t)i * n2 * K2, K2, n2, K2, BM, BKt)) return cudaErrorInvalidValue;
  const size_t smem = (size_t)NST * kStage4 + 1024 + 256;
  cudaError_t e = cudaFuncSetAttribute(syrk4_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  float* wh = reinterpret_cast<float*>(ws);
  float* wl = wh + (size_t)ntiles * BN * BM;
  Syrk4Args args{tiles_d, wh, wl, (int)(K2 / BKt), accumulate, err};
  syrk4_tc_kernel<<<ntiles, NT4, smem, st>>>(m[0], m[1], m[2], m[3], args);
  count_launch();
  return cudaGetLastError();
}

int mlgemm5_tc_nj_pad(int nj) { return (int)tc64::rup(nj, tc64::MBN); }
int mlgemm5_tc_kp(int rp) { return (int)tc64::rup(2 * (int64_t)rp, tc64::BKt); }
bool mlgemm5_tc_supported(int rp) { return rp > 0 && mlgemm5_tc_kp(rp) <= tc64::kMl5MaxK; }
size_t mlgemm5_tc_lslice_bytes(int nk, int rp, int nj) {
  return (size_t)tc64::NS5 * nk * mlgemm5_tc_nj_pad(nj) * mlgemm5_tc_kp(rp) * sizeof(__half) + 256;
}
size_t mlgemm5_tc_split_bytes(int64_t n2, int rp, int nq) {
  return (size_t)tc64::NS5 * nq * (2 * n2) * mlgemm5_tc_kp(rp) * sizeof(__half) + 256;
}

cudaError_t mlgemm5_tc_prepare(cudaStream_t st, const double2* L, const double* sw, int nk, int np, const int* perm,
                               const int* rank, int rp, int nj, void* lsl, int* col_exp) {
  const int Kp = mlgemm5_tc_kp(rp), njp = mlgemm5_tc_nj_pad(nj);
  if (njp % tc64::MBN != 0) return cudaErrorInvalidValue;
  const size_t per = (size_t)nk * njp * Kp;
  tc64::lslice5_kernel<<<dim3(njp, nk), 128, 0, st>>>(L, sw, np, perm, rank, nj, njp, Kp,
                                                       reinterpret_cast<__half*>(lsl), per, col_exp);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mlgemm5_tc_rowscale(cudaStream_t st, const ffcomplex* M, int64_t sq, int np, const int* qmap, int nS,
                                const int* perm, const int* rank, int rp, int64_t n2, int* row_exp) {
  if (n2 <= 0) return cudaSuccess;
  tc64::mrow_scale_ff_kernel<<<(unsigned)n2, 256, 0, st>>>(M, sq, np, qmap, nS, perm, rank, rp, row_exp);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mlgemm5_tc_chunk(cudaStream_t st, ffcomplex* M, int64_t sq, const int* qmap, int64_t n2, int np,
                             const int* perm, const int* rank, int rp, int nj, int j0, int nq, const int* row_exp,
                             void* split, const void* lsl, const int* col_exp, int nk, int* err) {
  using namespace tc64;
  if (n2 <= 0 || nq <= 0) return cudaSuccess;
  if (!mlgemm5_tc_supported(rp)) return cudaErrorInvalidValue;
  const int Kp = mlgemm5_tc_kp(rp), njp = mlgemm5_tc_nj_pad(nj);
  const size_t pa = (size_t)nq * (2 * n2) * Kp, pb = (size_t)nk * njp * Kp;
  __half* S = reinterpret_cast<__half*>(split);
  msplit5_kernel<<<nblk((int64_t)nq * n2 * (Kp / 2)), 256, 0, st>>>(M, sq, np, qmap, perm, rank, n2, j0, nq, Kp,
                                                                    row_exp, S, pa);
  count_launch();
  const __half* L1 = reinterpret_cast<const __half*>(lsl);
  CUtensorMap mA[NS5], mB[NS5];
  for (int i = 0; i < NS5; ++i)
    if (!make_map(&mA[i], S + i * pa, Kp, (int64_t)nq * 2 * n2, Kp, BM, BKt) ||
        !make_map(&mB[i], L1 + i * pb, Kp, (int64_t)nk * njp, Kp, MBN, BKt))
      return cudaErrorInvalidValue;
  const size_t smem = (size_t)NST * kStage5 + 1024 + 256;
  cudaError_t e = cudaFuncSetAttribute(mlgemm5_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int mt = (int)((2 * n2 + BM - 1) / BM), ntj = njp / MBN;
  Ml5Args args{M, qmap, row_exp, col_exp, sq, (int)n2, nj, njp, j0, Kp / BKt, err};
  mlgemm5_tc_kernel<<<dim3(mt * ntj, nq), NT5, smem, st>>>(mA[0], mA[1], mA[2], mA[3], mA[4], mB[0], mB[1], mB[2],
                                                            mB[3], mB[4], args);
  count_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------- V_xi on the tensor cores
// V_xi^q = Omega conj(c'^q) c'^q^T (Eq. 6) for the rx rows c'_I of the grid FFT of xi^q.
// With c' = a + i b, Re V_IJ = a_I.a_J + b_I.b_J and Im V_IJ = a_I.b_J - b_I.a_J, so one
// real SYRK of the 2 rxp rows  [a_I, b_I] (I < rxp)  and  [b_I, -a_I]  gives Re V in its
// leading block and -Im V in the block below it (rxp = rx rounded up to 128, padding
// rows zero).  It runs on syrk4_tc_kernel (four exact slices, the diagonal's left-out
// products added back), every q of a chunk a diagonal block of its own.
namespace tc64 {

// One block per stacked row r = (q, local): the row's exponent, its four slices over
// K2 columns (pairs (2G, 2G + 1)), and the sum of its left-out diagonal products.
__global__ void __launch_bounds__(256) vsplit_kernel(const ffcomplex* __restrict__ c, int64_t qs, int rx, int rxp,
                                                     int ng, int64_t K2, __half* __restrict__ S, int64_t per,
                                                     int* __restrict__ rowexp, double* __restrict__ corr) {
  const int64_t r = blockIdx.x;
  const int q = (int)(r / (2 * rxp)), loc = (int)(r % (2 * rxp)), I = loc % rxp;
  const bool lower = loc >= rxp;
  const ffcomplex* row = c + (int64_t)q * qs + (int64_t)I * ng;
  __shared__ float sm[32];
  float m = 0.f;
  if (I < rx)
    for (int g = threadIdx.x; g < ng; g += blockDim.x) m = fmaxf(m, amaxff(row[g]));
  m = block_max(m, sm);
  const int ex = slice_exp(m);
  double d = 0.0;
  for (int64_t c2 = threadIdx.x; c2 < K2 / 2; c2 += blockDim.x) {
    ffcomplex x{ffloat(0.f, 0.f), ffloat(0.f, 0.f)};
    if (I < rx && c2 < ng) x = row[c2];
    const ffloat u = lower ? x.y : x.x, w = lower ? -x.x : x.y;
    __half hu[NS4], hw[NS4];
    slice_ff<NS4>(u, ex, hu);
    slice_ff<NS4>(w, ex, hw);
    const int64_t at = r * K2 + 2 * c2;
#pragma unroll
    for (int i = 0; i < NS4; ++i) *reinterpret_cast<__half2*>(S + i * per + at) = __halves2half2(hu[i], hw[i]);
    const float u2 = __half2float(hu[1]), u3 = __half2float(hu[2]), u4 = __half2float(hu[3]);
    const float w2 = __half2float(hw[1]), w3 = __half2float(hw[2]), w4 = __half2float(hw[3]);
    const float t4 = 2.f * (u2 * u4 + w2 * w4) + (u3 * u3 + w3 * w3);
    const float t5 = 2.f * (u3 * u4 + w3 * w4), t6 = u4 * u4 + w4 * w4;
    d += (double)(t4 + (t5 + t6 * (1.f / 128.f)) * (1.f / 128.f)) * (1.0 / 268435456.0);
  }
  __shared__ double sd[8];
  for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) sd[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) t += sd[wi];
    corr[r] = t;
    rowexp[r] = ex;
  }
}

// V[q][I][J] = Omega (E'(I, J) - i E'(rxp + I, J)) of the q-th diagonal block, scaled back.
__global__ void vfinish_kernel(const float* __restrict__ wh, const float* __restrict__ wl,
                               const int* __restrict__ tile_of, int nt, int rx, int rxp, int nq,
                               const int* __restrict__ rowexp, const double* __restrict__ corr, double omega,
                               double2* __restrict__ V, int64_t ldv, int64_t vs) {
  const int64_t total = (int64_t)nq * rx * rx;
  auto val = [&](int64_t i, int64_t j) -> double {
    if (i < j) {
      const int64_t t = i;
      i = j;
      j = t;
    }
    const int t = tile_of[(i / BM) * nt + (j / BN)];
    const size_t idx = ((size_t)t * BN + (size_t)(j % BN)) * BM + (size_t)(i % BM);
    return (double)wh[idx] + (double)wl[idx];
  };
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e / ((int64_t)rx * rx)), I = (int)((e / rx) % rx), J = (int)(e % rx);
    const int64_t b = (int64_t)q * 2 * rxp;
    double re = val(b + I, b + J);
    if (I == J) re += corr[b + I];
    re *= ldexp(omega, -(rowexp[b + I] + rowexp[b + J]));
    const double im = -val(b + rxp + I, b + J) * ldexp(omega, -(rowexp[b + rxp + I] + rowexp[b + J]));
    V[(int64_t)q * vs + (int64_t)I * ldv + J] = make_double2(re, im);
  }
}

}  // namespace tc64

namespace {
struct VxiLayout {
  int rxp, nb;            // padded rows per half, 128-row blocks per half
  int64_t K2, rows;       // slice width, stacked rows of a chunk
  int tiles_per_q;
  size_t slices, ws, tiles, tile_of, rowexp, corr, total;
};
VxiLayout vxi_layout(int rx, int ng, int qc) {
  VxiLayout l;
  l.rxp = (int)tc64::rup(rx, 128);
  l.nb = l.rxp / 128;
  l.K2 = tc64::rup(2 * (int64_t)ng, tc64::BKt);
  l.rows = (int64_t)qc * 2 * l.rxp;
  l.tiles_per_q = l.nb * (l.nb + 1) / 2 + l.nb * l.nb;
  const int64_t nt = l.rows / 128;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  l.slices = al((size_t)tc64::NS4 * l.rows * l.K2 * sizeof(__half));
  l.ws = al((size_t)qc * l.tiles_per_q * 128 * 128 * 2 * sizeof(float));
  l.tiles = al((size_t)qc * l.tiles_per_q * sizeof(int2));
  l.tile_of = al((size_t)nt * nt * sizeof(int));
  l.rowexp = al((size_t)l.rows * sizeof(int));
  l.corr = al((size_t)l.rows * sizeof(double));
  l.total = l.slices + l.ws + l.tiles + l.tile_of + l.rowexp + l.corr;
  return l;
}
}  // namespace

int vxi_tc_chunk(int rx, int ng, size_t budget) {
  const size_t per_q = vxi_layout(rx, ng, 1).total;
  return (int)std::max<size_t>(1, std::min<size_t>(256, budget / std::max<size_t>(per_q, 1)));
}
size_t vxi_tc_work_bytes(int rx, int ng, int qc) { return vxi_layout(rx, ng, qc).total; }

cudaError_t vxi_tc(cudaStream_t st, const ffcomplex* c, int64_t qs, int rx, int ng, int nq, double omega,
                   double2* V, int64_t ldv, int64_t vs, void* work, int qc, int* err) {
  using namespace tc64;
  if (nq <= 0 || rx <= 0) return cudaSuccess;
  const VxiLayout l = vxi_layout(rx, ng, qc);
  uint8_t* w = reinterpret_cast<uint8_t*>(work);
  __half* S = reinterpret_cast<__half*>(w);
  void* ws = w + l.slices;
  int2* tiles_d = reinterpret_cast<int2*>(w + l.slices + l.ws);
  int* tof_d = reinterpret_cast<int*>(w + l.slices + l.ws + l.tiles);
  int* rowexp = reinterpret_cast<int*>(w + l.slices + l.ws + l.tiles + l.tile_of);
  double* corr = reinterpret_cast<double*>(w + l.slices + l.ws + l.tiles + l.tile_of + l.rowexp);
  for (int q0 = 0; q0 < nq; q0 += qc) {
    const int nc = std::min(qc, nq - q0);
    const int64_t rows = (int64_t)nc * 2 * l.rxp, nt = rows / 128;
    // tiles of each q's leading block (lower triangle) and of the block below it
    std::vector<int2> tl;
    std::vector<int> tof((size_t)(nt * nt), -1);
    for (int q = 0; q < nc; ++q) {
      const int b0 = q * 2 * l.nb;
      for (int ti = 0; ti < 2 * l.nb; ++ti)
        for (int tj = 0; tj < l.nb && tj <= ti; ++tj) {
          tof[(size_t)(b0 + ti) * nt + (b0 + tj)] = (int)tl.size();
          tl.push_back(make_int2(b0 + ti, b0 + tj));
        }
    }
    cudaError_t e = cudaMemcpyAsync(tiles_d, tl.data(), tl.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tof_d, tof.data(), tof.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    vsplit_kernel<<<(unsigned)rows, 256, 0, st>>>(c + (int64_t)q0 * qs, qs, rx, l.rxp, ng, l.K2, S, rows * l.K2,
                                                 rowexp, corr);
    count_launch();
    // the kernel's K2 is 2 nq nJ rounded to the k-block: nq = 1, nJ = ng
    e = syrk4_tc_mma(st, S, rows, 1, ng, tiles_d, (int)tl.size(), ws, 0, err);
    if (e != cudaSuccess) return e;
    const float* wh = reinterpret_cast<const float*>(ws);
    const float* wl = wh + tl.size() * 128 * 128;
    const int64_t tot = (int64_t)nc * rx * rx;
    int nbk = (int)std::min<int64_t>((tot + 255) / 256, 152 * 32);
    vfinish_kernel<<<std::max(nbk, 1), 256, 0, st>>>(wh, wl, tof_d, (int)nt, rx, l.rxp, nc, rowexp, corr, omega,
                                                    V + (int64_t)q0 * vs, ldv, vs);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace isdf
