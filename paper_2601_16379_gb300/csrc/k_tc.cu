// Tensor-core (tcgen05) kernels of the fragment ERIs, Eq. 19:
//     E = sum_q B^q B^q^H   with  B^q = M^q L^q   (V^q = L^q L^q^H).
// herk_tc_kernel forms E (below); mlgemm_tc_kernel forms B (further down, with
// four slices instead of three).
//
// Complex -> real: with B stored as interleaved (re, im) pairs, the real row
// P_a = (Re B_a0, Im B_a0, Re B_a1, ...) and Q_a = interleaved(-i B_a) give
//     Re E_ab = P_a . P_b      Im E_ab = Q_a . P_b,
// so one real GEMM D = A' B'^T with A' rows (P_0, Q_0, P_1, Q_1, ...) and
// B' = the P rows (every other row of A') yields both parts.  Only tiles that
// touch the lower triangle of the Hermitian E are computed.
//
// Precision (error-free slicing after Ozaki, Ogita, Oishi & Rump, 2012): each
// complex row a is scaled by a power of two 2^e_a so that its largest real
// component lies in [64, 128), and every scaled value is written as
//     v = s1 + s2/128 + s3/128^2 (+ remainder below 2^-15),  s_i integers, |s1| <= 128, |s2|, |s3| <= 64,
// stored as fp16 (exact).  The tcgen05.mma kind::f16 products of integer
// slices are integers, and the three weight groups
//     g0 = S1.T1,  g1 = S1.T2 + S2.T1,  g2 = S1.T3 + S2.T2 + S3.T1
// are accumulated in FP32 TMEM.  g0 carries weight 1 and must be exact: a
// chunk of 64 k-steps (1024 products of magnitude <= 2^14) keeps its partial
// sums integers of magnitude at most 2^24, so the FP32
// accumulation is exact whatever its rounding; g0 is double-buffered and each
// chunk is drained (overlapping the next chunk's MMAs) into a float-float
// (TwoSum) accumulator in global memory.  g1 and g2 carry weights 2^-7 and
// 2^-14, so the truncation of tcgen05's FP32 accumulation over longer runs
// enters only scaled down: they are drained every 4 and 16 chunks (bias below
// 1e-7 of |B_a||B_b|).  The result is accurate to ~2^-22 of |B_a||B_b|.
//
// Kernel roles (192 threads): warp 0 issues TMA loads, warp 1 allocates TMEM
// and issues the MMAs, warps 2-5 drain TMEM into the float-float workspace.
// Every wait is bounded: on expiry the CTA records an error code and exits.
#include <cuda.h>
#include <cuda_fp16.h>

#include <cstring>
#include <vector>

#include <algorithm>

#include "common.cuh"

namespace isdf {

namespace tc {

constexpr int BM = 128;        // A' rows per tile (64 complex rows of E)
constexpr int BN = 128;        // B' rows per tile (complex columns of E)
constexpr int BK = 64;         // fp16 per row per stage (one 128-byte swizzle row)
constexpr int STAGES = 2;
constexpr int NSLICE = 3;
constexpr int A_BYTES = BM * BK * 2;        // 16 KB per slice
constexpr int B_BYTES = BN * BK * 2;        // 16 KB per slice
constexpr int STAGE_BYTES = NSLICE * (A_BYTES + B_BYTES);  // 96 KB
constexpr int TMEM_COLS = 512;              // g0 (two buffers), g1, g2: four 128-column FP32 accumulators
constexpr int NTHREADS = 192;
constexpr int kChunkKB = 16;                // k-blocks per exact g0 chunk: 64 k-steps of 16
constexpr int kP1 = 4;                      // chunks per g1 drain
constexpr int kP2 = 16;                     // chunks per g2 drain
constexpr unsigned long long kWaitNs = 4000000000ULL;  // bounded waits: 4 s of device time

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase of parity `parity`; false on timeout or if another
// thread of the CTA already gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* s_err, int* g_err,
                                          int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0) {
      if (*s_err) return false;
      if (global_ns() - t0 > kWaitNs) break;
    }
  }
  *s_err = code;
  atomicCAS(g_err, 0, code);
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_sw128(const void* p) {
  const uint32_t a = smem_u32(p);
  return (uint64_t)((a & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

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

__global__ void __launch_bounds__(NTHREADS, 1)
    herk_tc_kernel(const __grid_constant__ CUtensorMap mA1, const __grid_constant__ CUtensorMap mA2,
                   const __grid_constant__ CUtensorMap mA3, const __grid_constant__ CUtensorMap mB1,
                   const __grid_constant__ CUtensorMap mB2, const __grid_constant__ CUtensorMap mB3, TileArgs args) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment of the shared-window address (128-byte swizzle atoms)
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* full = bars;                   // [STAGES]
  uint64_t* empty = bars + STAGES;         // [STAGES]
  uint64_t* accf = bars + 2 * STAGES;      // [2] chunk accumulated (per g0 buffer)
  uint64_t* acce = bars + 2 * STAGES + 2;  // [2] g0 buffer drained
  uint64_t* acce1 = bars + 2 * STAGES + 4; // g1 drained
  uint64_t* acce2 = bars + 2 * STAGES + 5; // g2 drained
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 6);
  volatile int* s_err = reinterpret_cast<volatile int*>(s_tmem + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int2 tile = args.tiles[blockIdx.x];
  const int nkb = args.nkb;
  const int nchunks = (nkb + kChunkKB - 1) / kChunkKB;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 128);
    }
    mbar_init(acce1, 128);
    mbar_init(acce2, 128);
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
      const CUtensorMap* ma[3] = {&mA1, &mA2, &mA3};
      const CUtensorMap* mb[3] = {&mB1, &mB2, &mB3};
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % STAGES, r = kb / STAGES;
        if (!mbar_wait(&empty[s], (r & 1) ^ 1, s_err, args.err, 1)) break;
        uint8_t* st = smem + s * STAGE_BYTES;
        mbar_expect_tx(&full[s], STAGE_BYTES);
        const int x = kb * BK;
#pragma unroll
        for (int i = 0; i < NSLICE; ++i) {
          tma_load_2d(st + i * A_BYTES, ma[i], &full[s], x, tile.x * BM);
          tma_load_2d(st + NSLICE * A_BYTES + i * B_BYTES, mb[i], &full[s], x, tile.y * BN);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % STAGES, r = kb / STAGES;
        const int c = kb / kChunkKB;
        const bool first_in_chunk = (kb % kChunkKB) == 0;
        const bool reset1 = first_in_chunk && (c % kP1) == 0;
        const bool reset2 = first_in_chunk && (c % kP2) == 0;
        if (first_in_chunk) {
          bool ok = true;
          // g0 buffer (c & 1) was last used by chunk c - 2
          if (c >= 2) ok = mbar_wait(&acce[c & 1], ((c >> 1) - 1) & 1, s_err, args.err, 2);
          if (ok && reset1 && c > 0) ok = mbar_wait(acce1, ((c / kP1) - 1) & 1, s_err, args.err, 5);
          if (ok && reset2 && c > 0) ok = mbar_wait(acce2, ((c / kP2) - 1) & 1, s_err, args.err, 6);
          if (!ok) break;
          tc_fence_after();
        }
        if (!mbar_wait(&full[s], r & 1, s_err, args.err, 3)) break;
        tc_fence_after();
        const uint8_t* st = smem + s * STAGE_BYTES;
        uint64_t dA[3], dB[3];
#pragma unroll
        for (int i = 0; i < NSLICE; ++i) {
          dA[i] = sdesc_sw128(st + i * A_BYTES);
          dB[i] = sdesc_sw128(st + NSLICE * A_BYTES + i * B_BYTES);
        }
        const uint32_t g0 = tmem_base + (uint32_t)((c & 1) * BN), g1 = tmem_base + 2 * BN,
                       g2 = tmem_base + 3 * BN;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t off = (uint64_t)(kk * 32) >> 4;  // 16 fp16 = 32 bytes along K
          const uint32_t a0 = (first_in_chunk && kk == 0) ? 0u : 1u;
          const uint32_t a1 = (reset1 && kk == 0) ? 0u : 1u;
          const uint32_t a2 = (reset2 && kk == 0) ? 0u : 1u;
          umma_f16(g0, dA[0] + off, dB[0] + off, kIdesc, a0);
          umma_f16(g1, dA[0] + off, dB[1] + off, kIdesc, a1);
          umma_f16(g1, dA[1] + off, dB[0] + off, kIdesc, 1u);
          umma_f16(g2, dA[0] + off, dB[2] + off, kIdesc, a2);
          umma_f16(g2, dA[1] + off, dB[1] + off, kIdesc, 1u);
          umma_f16(g2, dA[2] + off, dB[0] + off, kIdesc, 1u);
        }
        umma_commit(&empty[s]);
        if ((kb % kChunkKB) == kChunkKB - 1 || kb == nkb - 1) umma_commit(&accf[c & 1]);
      }
    }
  } else {
    // epilogue: warps 2..5 -> TMEM lane quarter (warp % 4)
    const int q = warp & 3;
    const int row = q * 32 + lane;
    float* __restrict__ wh = args.ws_hi + (size_t)blockIdx.x * BN * BM;
    float* __restrict__ wl = args.ws_lo + (size_t)blockIdx.x * BN * BM;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    for (int c = 0; c < nchunks; ++c) {
      if (!mbar_wait(&accf[c & 1], (c >> 1) & 1, s_err, args.err, 4)) break;
      tc_fence_after();
      const bool last = (c == nchunks - 1);
      const bool drain1 = last || (c % kP1) == kP1 - 1;
      const bool drain2 = last || (c % kP2) == kP2 - 1;
#pragma unroll 1
      for (int cb = 0; cb < BN / 32; ++cb) {
        uint32_t v0[32];
        float H[32], L[32];
        const size_t base = (size_t)(cb * 32) * BM + row;
        const bool fresh = (c == 0) && !args.accumulate;
        if (!fresh) {
          // issue all 64 global loads of this column block before the TMEM reads
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            H[j] = wh[base + (size_t)j * BM];
            L[j] = wl[base + (size_t)j * BM];
          }
        }
        tmem_ld32(tmem_base + lane_off + (uint32_t)((c & 1) * BN + cb * 32), v0);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float a0 = __uint_as_float(v0[j]);
          if (fresh) {
            H[j] = a0;
            L[j] = 0.f;
          } else {
            // (H, L) += a0 with TwoSum on the high part
            const float S = H[j] + a0;
            const float bp = S - H[j];
            const float e = (H[j] - (S - bp)) + (a0 - bp);
            H[j] = S;
            L[j] += e;
          }
        }
        if (drain1) {
          uint32_t v1[32];
          tmem_ld32(tmem_base + lane_off + (uint32_t)(2 * BN + cb * 32), v1);
#pragma unroll
          for (int j = 0; j < 32; ++j) L[j] = fmaf(__uint_as_float(v1[j]), 1.0f / 128.0f, L[j]);
        }
        if (drain2) {
          uint32_t v2[32];
          tmem_ld32(tmem_base + lane_off + (uint32_t)(3 * BN + cb * 32), v2);
#pragma unroll
          for (int j = 0; j < 32; ++j) L[j] = fmaf(__uint_as_float(v2[j]), 1.0f / 16384.0f, L[j]);
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          wh[base + (size_t)j * BM] = H[j];
          wl[base + (size_t)j * BM] = L[j];
        }
      }
      tc_fence_before();
      mbar_arrive(&acce[c & 1]);
      if (drain1) mbar_arrive(acce1);
      if (drain2) mbar_arrive(acce2);
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

// Per complex row a: exponent e_a with max_k max(|Re B_ak|, |Im B_ak|) 2^e_a in [64, 128).
__global__ void row_scale_kernel(BView B, int64_t n2, int64_t K, int* __restrict__ row_exp) {
  const int64_t a = blockIdx.x;
  if (a >= n2) return;
  float m = 0.f;
  for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
    const float2 v = B.at(a, k);
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  __shared__ float sm[32];
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mm = fmaxf(mm, sm[i]);
    row_exp[a] = (mm > 0.f && isfinite(mm)) ? 6 - ilogbf(mm) : 0;
  }
}

// Slices of A': row 2a = P_a (Re, Im interleaved), row 2a+1 = Q_a (Im, -Re); columns
// beyond 2K are zero.  v = x 2^e_a = s1 + s2/128 + s3/128^2 (+ remainder).
__global__ void split_kernel(BView B, int64_t n2, int64_t k0, int64_t K, int64_t K2,
                             const int* __restrict__ row_exp, __half* __restrict__ S1, __half* __restrict__ S2,
                             __half* __restrict__ S3) {
  const int64_t total = n2 * (K2 / 2);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / (K2 / 2), k = e % (K2 / 2);
    float2 v = make_float2(0.f, 0.f);
    if (k < K) v = B.at(a, k0 + k);
    const int ex = row_exp[a];
    const float pr = ldexpf(v.x, ex), pi = ldexpf(v.y, ex);
    const float vals[4] = {pr, pi, pi, -pr};
    __half h1[4], h2[4], h3[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float s1 = rintf(vals[t]);
      const float r1 = (vals[t] - s1) * 128.f;
      const float s2 = rintf(r1);
      const float r2 = (r1 - s2) * 128.f;
      const float s3 = rintf(r2);
      h1[t] = __float2half_rn(s1);
      h2[t] = __float2half_rn(s2);
      h3[t] = __float2half_rn(s3);
    }
    const int64_t rP = (2 * a) * K2 + 2 * k, rQ = (2 * a + 1) * K2 + 2 * k;
    *reinterpret_cast<__half2*>(S1 + rP) = __halves2half2(h1[0], h1[1]);
    *reinterpret_cast<__half2*>(S2 + rP) = __halves2half2(h2[0], h2[1]);
    *reinterpret_cast<__half2*>(S3 + rP) = __halves2half2(h3[0], h3[1]);
    *reinterpret_cast<__half2*>(S1 + rQ) = __halves2half2(h1[2], h1[3]);
    *reinterpret_cast<__half2*>(S2 + rQ) = __halves2half2(h2[2], h2[3]);
    *reinterpret_cast<__half2*>(S3 + rQ) = __halves2half2(h3[2], h3[3]);
  }
}

// E (complex128, n2 x n2, Hermitian) from the float-float tile workspace,
// scaled by scale * 2^-(e_a + e_b).
__global__ void herk_finish_kernel(const float* __restrict__ wh, const float* __restrict__ wl,
                                   const int2* __restrict__ tiles, int ntiles, int64_t n2,
                                   const int* __restrict__ row_exp, double scale, double2* __restrict__ E) {
  const int64_t per = (int64_t)BN * (BM / 2);
  const int64_t total = per * ntiles;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / per);
    const int c = (int)((e % per) / (BM / 2));
    const int al = (int)(e % (BM / 2));
    const int64_t a = (int64_t)tiles[t].x * (BM / 2) + al;
    const int64_t b = (int64_t)tiles[t].y * BN + c;
    if (a >= n2 || b >= n2 || a < b) continue;
    const size_t base = ((size_t)t * BN + c) * BM;
    const double f = ldexp(scale, -(row_exp[a] + row_exp[b]));
    const double re = ((double)wh[base + 2 * al] + (double)wl[base + 2 * al]) * f;
    const double im = ((double)wh[base + 2 * al + 1] + (double)wl[base + 2 * al + 1]) * f;
    E[a * n2 + b] = make_double2(re, im);
    if (a != b) E[b * n2 + a] = make_double2(re, -im);
  }
}

// ---------------------------------------------------------------------------
// B^q = M^q L^q on the tensor cores with four exact slices.
//
// Real form: A' rows P_a = (Re M_aI, Im M_aI)_I and Q_a = interleaved(-i M_a),
// B' rows R_J = (Re L_IJ, -Im L_IJ)_I, so (A' R_J)[P_a] = Re B_aJ and
// (A' R_J)[Q_a] = Im B_aJ.  M rows are scaled by 2^e_a (largest component of
// M_a over the q of the sum in [64, 128)), L columns by 2^f_qJ per q; both are
// cut into four integer slices v = s1 + s2/128 + s3/128^2 + s4/128^3 (28 bits:
// B = M W^T L_xi carries the cancellation of the ill-conditioned W, and three
// slices, 21 bits, measurably degrade the traces).  Ten fp16 products feed four
// weight groups
//   g0 = S1T1, g1 = S1T2 + S2T1, g2 = S1T3 + S2T2 + S3T1,
//   g3 = S1T4 + S2T3 + S3T2 + S4T1;
// with K' = 2 N_P <= kMlMaxK every partial sum of each group is an integer of
// magnitude below 2^24 (g3: at most 3 * 2^13 per k), so the FP32 TMEM
// accumulation is exact; the epilogue forms g0 + g1/2^7 + g2/2^14 + g3/2^21
// once and rescales.
constexpr int MSL = 4;                                     // slices per operand
constexpr int MBN = 96;                                    // output columns per tile (N of the MMA)
constexpr int MB_BYTES = MBN * BK * 2;                     // 12 KB per slice
constexpr int MSTAGE_BYTES = MSL * (A_BYTES + MB_BYTES);   // 112 KB
constexpr int kMlMaxK = 640;                               // K' bound for exact accumulation
constexpr uint32_t kIdescMl = (1u << 4) | ((uint32_t)(MBN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

struct MlArgs {
  float2* out;          // B: element (a, J) of the chunk's q-point ql at out[slot sq + a np + J]
  const int* qmap;      // slot of the chunk's q-points (indexed j0 + ql)
  const int* row_exp;   // e_a, [n2]
  const int* col_exp;   // f_qJ, [Nk][np_pad] indexed by slot
  int64_t sq;           // q stride of out
  int n2, np, np_pad, j0, nkb;
  int* err;
};

__global__ void __launch_bounds__(NTHREADS, 1)
    mlgemm_tc_kernel(const __grid_constant__ CUtensorMap mA1, const __grid_constant__ CUtensorMap mA2,
                     const __grid_constant__ CUtensorMap mA3, const __grid_constant__ CUtensorMap mA4,
                     const __grid_constant__ CUtensorMap mB1, const __grid_constant__ CUtensorMap mB2,
                     const __grid_constant__ CUtensorMap mB3, const __grid_constant__ CUtensorMap mB4, MlArgs args) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * MSTAGE_BYTES);
  uint64_t* full = bars;               // [STAGES]
  uint64_t* empty = bars + STAGES;     // [STAGES]
  uint64_t* accf = bars + 2 * STAGES;  // accumulation finished
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  volatile int* s_err = reinterpret_cast<volatile int*>(s_tmem + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = (2 * args.n2 + BM - 1) / BM;
  const int ti = blockIdx.x % mt, tj = blockIdx.x / mt, ql = blockIdx.y;
  const int slot = args.qmap ? args.qmap[args.j0 + ql] : args.j0 + ql;
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
      const CUtensorMap* ma[MSL] = {&mA1, &mA2, &mA3, &mA4};
      const CUtensorMap* mb[MSL] = {&mB1, &mB2, &mB3, &mB4};
      const int arow = ql * 2 * args.n2 + ti * BM, brow = slot * args.np_pad + tj * MBN;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % STAGES, r = kb / STAGES;
        if (!mbar_wait(&empty[s], (r & 1) ^ 1, s_err, args.err, 11)) break;
        uint8_t* st = smem + s * MSTAGE_BYTES;
        mbar_expect_tx(&full[s], MSTAGE_BYTES);
        const int x = kb * BK;
#pragma unroll
        for (int i = 0; i < MSL; ++i) {
          tma_load_2d(st + i * A_BYTES, ma[i], &full[s], x, arow);
          tma_load_2d(st + MSL * A_BYTES + i * MB_BYTES, mb[i], &full[s], x, brow);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t g0 = tmem_base, g1 = tmem_base + MBN, g2 = tmem_base + 2 * MBN, g3 = tmem_base + 3 * MBN;
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
          dA[i] = sdesc_sw128(st + i * A_BYTES);
          dB[i] = sdesc_sw128(st + MSL * A_BYTES + i * MB_BYTES);
        }
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t off = (uint64_t)(kk * 32) >> 4;
          const uint32_t acc = (kb == 0 && kk == 0) ? 0u : 1u;
          umma_f16(g0, dA[0] + off, dB[0] + off, kIdescMl, acc);
          umma_f16(g1, dA[0] + off, dB[1] + off, kIdescMl, acc);
          umma_f16(g1, dA[1] + off, dB[0] + off, kIdescMl, 1u);
          umma_f16(g2, dA[0] + off, dB[2] + off, kIdescMl, acc);
          umma_f16(g2, dA[1] + off, dB[1] + off, kIdescMl, 1u);
          umma_f16(g2, dA[2] + off, dB[0] + off, kIdescMl, 1u);
          umma_f16(g3, dA[0] + off, dB[3] + off, kIdescMl, acc);
          umma_f16(g3, dA[1] + off, dB[2] + off, kIdescMl, 1u);
          umma_f16(g3, dA[2] + off, dB[1] + off, kIdescMl, 1u);
          umma_f16(g3, dA[3] + off, dB[0] + off, kIdescMl, 1u);
        }
        umma_commit(&empty[s]);
      }
      if (ok) umma_commit(accf);
    }
  } else {
    // epilogue: warps 2..5 -> TMEM lane quarter (warp % 4); rows P_a / Q_a are lanes 2i / 2i+1
    const int q = warp & 3;
    const int r = q * 32 + lane;            // row of the tile
    const int64_t R = (int64_t)ti * BM + r;  // row of A'
    const int al = r >> 1, part = r & 1;
    const int64_t a = R >> 1;
    // warp-uniform, so that the .sync.aligned TMEM loads are taken by whole warps
    const bool okw = __all_sync(0xffffffffu, mbar_wait(accf, 0, s_err, args.err, 13));
    tc_fence_after();
    // the operand stages are idle now: stage the 64 x MBN complex tile for coalesced stores
    constexpr int kPitch = 2 * MBN + 2;     // floats per staged row (bank-conflict padding)
    float* tileS = reinterpret_cast<float*>(smem);
    const int ea = (okw && a < args.n2) ? args.row_exp[a] : 0;
    const int* fcol = args.col_exp + (int64_t)slot * args.np_pad + tj * MBN;
#pragma unroll 1
    for (int cb = 0; cb < MBN / 32; ++cb) {
      uint32_t v0[32] = {}, v1[32] = {}, v2[32] = {}, v3[32] = {};
      if (okw) {
        const uint32_t lo = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(cb * 32);
        tmem_ld32(lo, v0);
        tmem_ld32(lo + MBN, v1);
        tmem_ld32(lo + 2 * MBN, v2);
        tmem_ld32(lo + 3 * MBN, v3);
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float v = __uint_as_float(v0[j]) +
                        (__uint_as_float(v1[j]) * (1.0f / 128.0f) +
                         (__uint_as_float(v2[j]) * (1.0f / 16384.0f) + __uint_as_float(v3[j]) * (1.0f / 2097152.0f)));
        const int Jl = cb * 32 + j;
        tileS[al * kPitch + 2 * Jl + part] = ldexpf(v, -(ea + fcol[Jl]));
      }
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (okw) {
      const int t = threadIdx.x - 64;
      float2* outq = args.out + (int64_t)slot * args.sq;
      for (int idx = t; idx < (BM / 2) * MBN; idx += 128) {
        const int ar = idx / MBN, Jl = idx % MBN;
        const int64_t aa = (int64_t)ti * (BM / 2) + ar;
        const int J = tj * MBN + Jl;
        if (aa < args.n2 && J < args.np)
          outq[aa * args.np + J] = *reinterpret_cast<const float2*>(tileS + ar * kPitch + 2 * Jl);
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

__device__ __forceinline__ float round_int(float x) { return rintf(x); }
__device__ __forceinline__ double round_int(double x) { return rint(x); }

// Four integer slices of v (|v| < 128): v = s1 + s2/128 + s3/128^2 + s4/128^3 + r.
template <typename R>
__device__ __forceinline__ void slice4(R v, __half& h1, __half& h2, __half& h3, __half& h4) {
  const R s1 = round_int(v);
  const R r1 = (v - s1) * (R)128;
  const R s2 = round_int(r1);
  const R r2 = (r1 - s2) * (R)128;
  const R s3 = round_int(r2);
  const R r3 = (r2 - s3) * (R)128;
  h1 = __float2half_rn((float)s1);
  h2 = __float2half_rn((float)s2);
  h3 = __float2half_rn((float)s3);
  h4 = __float2half_rn((float)round_int(r3));
}

// A' slices of M for the q-points j0..j0+nq-1 of the sum: block ql holds rows
// 2a (P_a) and 2a+1 (Q_a) over Kp columns, zero beyond 2 np.
__global__ void msplit_kernel(BView M, int64_t n2, int np, int j0, int nq, int Kp, const int* __restrict__ row_exp,
                              __half* __restrict__ S1, __half* __restrict__ S2, __half* __restrict__ S3,
                              __half* __restrict__ S4) {
  const int64_t half = Kp / 2, total = (int64_t)nq * n2 * half;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ql = e / (n2 * half), rem = e % (n2 * half);
    const int64_t a = rem / half, k = rem % half;
    float2 v = make_float2(0.f, 0.f);
    if (k < np) v = M.at(a, (int64_t)(j0 + ql) * np + k);
    const int ex = row_exp[a];
    const float pr = ldexpf(v.x, ex), pi = ldexpf(v.y, ex);
    const float vals[4] = {pr, pi, pi, -pr};
    __half h1[4], h2[4], h3[4], h4[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) slice4<float>(vals[t], h1[t], h2[t], h3[t], h4[t]);
    const int64_t rP = (ql * 2 * n2 + 2 * a) * Kp + 2 * k, rQ = rP + Kp;
    *reinterpret_cast<__half2*>(S1 + rP) = __halves2half2(h1[0], h1[1]);
    *reinterpret_cast<__half2*>(S2 + rP) = __halves2half2(h2[0], h2[1]);
    *reinterpret_cast<__half2*>(S3 + rP) = __halves2half2(h3[0], h3[1]);
    *reinterpret_cast<__half2*>(S4 + rP) = __halves2half2(h4[0], h4[1]);
    *reinterpret_cast<__half2*>(S1 + rQ) = __halves2half2(h1[2], h1[3]);
    *reinterpret_cast<__half2*>(S2 + rQ) = __halves2half2(h2[2], h2[3]);
    *reinterpret_cast<__half2*>(S3 + rQ) = __halves2half2(h3[2], h3[3]);
    *reinterpret_cast<__half2*>(S4 + rQ) = __halves2half2(h4[2], h4[3]);
  }
}

// B' slices of w_q^{1/2} L^q: block (q, J) is the row R_J = (Re L_IJ, -Im L_IJ)_I
// scaled by 2^f_qJ (largest component in [64, 128)), rows J >= np and columns
// beyond 2 np zero.  Layout [q][np_pad][Kp] per slice; exponents [q][np_pad].
__global__ void lslice_kernel(const double2* __restrict__ L, const double* __restrict__ sw, int np, int np_pad,
                              int Kp, __half* __restrict__ S1, __half* __restrict__ S2, __half* __restrict__ S3,
                              __half* __restrict__ S4, int* __restrict__ col_exp) {
  const int q = blockIdx.y, J = blockIdx.x;
  const double w = sw[q];
  const double2* Lq = L + (int64_t)q * np * np;
  double m = 0.0;
  if (J < np)
    for (int I = threadIdx.x; I < np; I += blockDim.x) {
      const double2 v = Lq[(int64_t)I * np + J];
      m = fmax(m, fmax(fabs(v.x * w), fabs(v.y * w)));
    }
  __shared__ double sm[32];
  __shared__ int s_e;
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mm = fmax(mm, sm[i]);
    s_e = (mm > 0.0 && isfinite(mm)) ? 6 - ilogb(mm) : 0;
    col_exp[(int64_t)q * np_pad + J] = s_e;
  }
  __syncthreads();
  const int ex = s_e;
  const int64_t row = ((int64_t)q * np_pad + J) * Kp;
  for (int k = threadIdx.x; k < Kp / 2; k += blockDim.x) {
    double re = 0.0, im = 0.0;
    if (J < np && k < np) {
      const double2 v = Lq[(int64_t)k * np + J];
      re = ldexp(v.x * w, ex);
      im = -ldexp(v.y * w, ex);
    }
    __half a1, a2, a3, a4, b1, b2, b3, b4;
    slice4<double>(re, a1, a2, a3, a4);
    slice4<double>(im, b1, b2, b3, b4);
    *reinterpret_cast<__half2*>(S1 + row + 2 * k) = __halves2half2(a1, b1);
    *reinterpret_cast<__half2*>(S2 + row + 2 * k) = __halves2half2(a2, b2);
    *reinterpret_cast<__half2*>(S3 + row + 2 * k) = __halves2half2(a3, b3);
    *reinterpret_cast<__half2*>(S4 + row + 2 * k) = __halves2half2(a4, b4);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D fp16 map: rows of `inner` elements, row pitch `pitch_elems`, box (BK x box_rows), 128-byte swizzle.
bool make_map(CUtensorMap* m, const __half* base, int64_t inner, int64_t rows, int64_t pitch_elems, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(pitch_elems * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

inline int nblk(int64_t total) {
  int64_t nb = (total + 255) / 256;
  if (nb > 152 * 32) nb = 152 * 32;
  return nb < 1 ? 1 : (int)nb;
}

}  // namespace tc

size_t herk_tc_split_bytes(int64_t n2, int64_t K) {
  const int64_t K2 = ((2 * K + tc::BK - 1) / tc::BK) * tc::BK;
  return (size_t)tc::NSLICE * (2 * n2) * K2 * sizeof(__half) + 256;
}

// Lower-triangle tiles in launch order.  Every CTA streams the whole K extent of
// its A' and B' rows, and about one CTA per SM is resident, so the order decides
// what L2 can share: tiles go in bands of kGroupA A'-tiles, and within a band
// column by column, so that the ~150 CTAs of a wave read about 12 A'-blocks and
// 12 B'-blocks instead of ~150 different A'-blocks.
void herk_tc_tiles(int64_t n2, std::vector<int2>& tiles) {
  constexpr int64_t kGroupA = 12;
  tiles.clear();
  const int64_t mt = (2 * n2 + tc::BM - 1) / tc::BM, nt = (n2 + tc::BN - 1) / tc::BN;
  for (int64_t t0 = 0; t0 < mt; t0 += kGroupA)
    for (int64_t tj = 0; tj < nt; ++tj)
      for (int64_t ti = t0; ti < std::min(mt, t0 + kGroupA); ++ti)
        if (ti * (tc::BM / 2) + (tc::BM / 2 - 1) >= tj * tc::BN) tiles.push_back(make_int2((int)ti, (int)tj));
}

size_t herk_tc_ws_bytes(int64_t ntiles) { return (size_t)ntiles * tc::BN * tc::BM * 2 * sizeof(float); }

// Row exponents over the whole row: element (a, k) = B[slot(Q) sQ + a sA + J], k = Q nJ + J < K.
cudaError_t herk_tc_rowscale(cudaStream_t st, const float2* B, int64_t sQ, int64_t sA, int64_t nJ, const int* qmap,
                             int64_t n2, int64_t K, int* row_exp) {
  tc::BView bv{B, sQ, sA, nJ, qmap};
  tc::row_scale_kernel<<<(unsigned)n2, 256, 0, st>>>(bv, n2, K, row_exp);
  count_launch();
  return cudaGetLastError();
}

// ws (+)= slices of columns [k0, k0 + Kc) of B: one K chunk of E = B B^H.
cudaError_t herk_tc_chunk(cudaStream_t st, const float2* B, int64_t sQ, int64_t sA, int64_t nJ, const int* qmap,
                          int64_t n2, int64_t k0, int64_t Kc, const int* row_exp, void* split, const int2* tiles_d,
                          int ntiles, void* ws, int accumulate, int* err) {
  using namespace tc;
  if (n2 <= 0 || Kc <= 0 || ntiles <= 0) return cudaSuccess;
  const int64_t K2 = ((2 * Kc + BK - 1) / BK) * BK;
  __half* S1 = reinterpret_cast<__half*>(split);
  __half* S2 = S1 + (size_t)(2 * n2) * K2;
  __half* S3 = S2 + (size_t)(2 * n2) * K2;
  BView bv{B, sQ, sA, nJ, qmap};
  split_kernel<<<nblk(n2 * (K2 / 2)), 256, 0, st>>>(bv, n2, k0, Kc, K2, row_exp, S1, S2, S3);
  count_launch();
  CUtensorMap mA[3], mB[3];
  __half* sl[3] = {S1, S2, S3};
  for (int i = 0; i < 3; ++i)
    if (!make_map(&mA[i], sl[i], K2, 2 * n2, K2, BM) || !make_map(&mB[i], sl[i], K2, n2, 2 * K2, BN))
      return cudaErrorInvalidValue;
  const size_t smem = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
  cudaError_t e = cudaFuncSetAttribute(herk_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  float* wh = reinterpret_cast<float*>(ws);
  float* wl = wh + (size_t)ntiles * BN * BM;
  TileArgs args{tiles_d, wh, wl, (int)(K2 / BK), accumulate, err};
  herk_tc_kernel<<<ntiles, NTHREADS, smem, st>>>(mA[0], mA[1], mA[2], mB[0], mB[1], mB[2], args);
  count_launch();
  return cudaGetLastError();
}

// E (complex128 n2 x n2, full Hermitian) = scale * 2^-(e_a + e_b) * workspace.
cudaError_t herk_tc_finish(cudaStream_t st, const void* ws, const int2* tiles_d, int ntiles, int64_t n2,
                           const int* row_exp, double scale, double2* E) {
  using namespace tc;
  const float* wh = reinterpret_cast<const float*>(ws);
  const float* wl = wh + (size_t)ntiles * BN * BM;
  herk_finish_kernel<<<nblk((int64_t)ntiles * BN * (BM / 2)), 256, 0, st>>>(wh, wl, tiles_d, ntiles, n2, row_exp,
                                                                            scale, E);
  count_launch();
  return cudaGetLastError();
}

// One-shot E = scale * B B^H for B complex64 n2 x K with row pitch ldb.
cudaError_t herk_tc(cudaStream_t st, const float2* B, int64_t n2, int64_t K, int64_t ldb, double scale,
                    void* split, const int2* tiles_d, int ntiles, void* ws, int* row_exp, int* err, double2* E) {
  cudaError_t e = herk_tc_rowscale(st, B, 0, ldb, K, nullptr, n2, K, row_exp);
  if (e != cudaSuccess) return e;
  e = herk_tc_chunk(st, B, 0, ldb, K, nullptr, n2, 0, K, row_exp, split, tiles_d, ntiles, ws, 0, err);
  if (e != cudaSuccess) return e;
  return herk_tc_finish(st, ws, tiles_d, ntiles, n2, row_exp, scale, E);
}

// ---- B = M L on the tensor cores, four slices (host side)
int mlgemm_tc_kp(int np) { return ((2 * np + tc::BK - 1) / tc::BK) * tc::BK; }
int mlgemm_tc_np_pad(int np) { return ((np + tc::MBN - 1) / tc::MBN) * tc::MBN; }
bool mlgemm_tc_supported(int np) { return np > 0 && mlgemm_tc_kp(np) <= tc::kMlMaxK; }
size_t mlgemm_tc_lslice_bytes(int nk, int np) {
  return (size_t)tc::MSL * nk * mlgemm_tc_np_pad(np) * mlgemm_tc_kp(np) * sizeof(__half) + 256;
}
size_t mlgemm_tc_split_bytes(int64_t n2, int np, int nq) {
  return (size_t)tc::MSL * nq * (2 * n2) * mlgemm_tc_kp(np) * sizeof(__half) + 256;
}

cudaError_t mlgemm_tc_prepare(cudaStream_t st, const double2* L, const double* sw, int nk, int np, void* lsl,
                              int* col_exp) {
  using namespace tc;
  const int Kp = mlgemm_tc_kp(np), npp = mlgemm_tc_np_pad(np);
  const size_t per = (size_t)nk * npp * Kp;
  __half* S1 = reinterpret_cast<__half*>(lsl);
  lslice_kernel<<<dim3(npp, nk), 128, 0, st>>>(L, sw, np, npp, Kp, S1, S1 + per, S1 + 2 * per, S1 + 3 * per,
                                                col_exp);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mlgemm_tc_chunk(cudaStream_t st, float2* M, int64_t sq, const int* qmap, int64_t n2, int np, int j0,
                            int nq, const int* row_exp, void* split, const void* lsl, const int* col_exp, int nk,
                            int* err) {
  using namespace tc;
  if (n2 <= 0 || nq <= 0) return cudaSuccess;
  if (!mlgemm_tc_supported(np)) return cudaErrorInvalidValue;
  const int Kp = mlgemm_tc_kp(np), npp = mlgemm_tc_np_pad(np);
  const size_t pa = (size_t)nq * (2 * n2) * Kp, pb = (size_t)nk * npp * Kp;
  __half* S1 = reinterpret_cast<__half*>(split);
  BView mv{M, sq, np, np, qmap};
  msplit_kernel<<<nblk((int64_t)nq * n2 * (Kp / 2)), 256, 0, st>>>(mv, n2, np, j0, nq, Kp, row_exp, S1, S1 + pa,
                                                                   S1 + 2 * pa, S1 + 3 * pa);
  count_launch();
  const __half* L1 = reinterpret_cast<const __half*>(lsl);
  CUtensorMap mA[MSL], mB[MSL];
  for (int i = 0; i < MSL; ++i)
    if (!make_map(&mA[i], S1 + i * pa, Kp, (int64_t)nq * 2 * n2, Kp, BM) ||
        !make_map(&mB[i], L1 + i * pb, Kp, (int64_t)nk * npp, Kp, MBN))
      return cudaErrorInvalidValue;
  const size_t smem = (size_t)STAGES * MSTAGE_BYTES + 1024 + 256;
  cudaError_t e = cudaFuncSetAttribute(mlgemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int mt = (int)((2 * n2 + BM - 1) / BM), ntj = npp / MBN;
  MlArgs args{M, qmap, row_exp, col_exp, sq, (int)n2, np, npp, j0, Kp / BK, err};
  mlgemm_tc_kernel<<<dim3(mt * ntj, nq), NTHREADS, smem, st>>>(mA[0], mA[1], mA[2], mA[3], mB[0], mB[1], mB[2],
                                                                mB[3], args);
  count_launch();
  return cudaGetLastError();
}

}  // namespace isdf
