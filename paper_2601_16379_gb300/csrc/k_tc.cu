// Tensor-core (tcgen05) contraction of the fragment ERIs, Eq. 19:
//     E = sum_q B^q B^q^H   with  B^q = M^q L^q   (V^q = L^q L^q^H).
//
// Complex -> real: with B stored as interleaved (re, im) pairs, the real row
// P_a = (Re B_a0, Im B_a0, Re B_a1, ...) and Q_a = interleaved(-i B_a) give
//     Re E_ab = P_a . P_b      Im E_ab = Q_a . P_b,
// so one real GEMM D = A' B'^T with A' rows (P_0, Q_0, P_1, Q_1, ...) and
// B' = the P rows (every other row of A') yields both parts.  Only tiles that
// touch the lower triangle of the Hermitian E are computed.
//
// Precision: every real value is split as x = hi + lo with hi = fp16(s x) and
// lo = fp16(s x - hi) (s a power of two), and D = Ah Bh^T + Ah Bl^T + Al Bh^T
// is accumulated by tcgen05.mma kind::f16 in FP32 TMEM.  The accumulator is
// flushed every `flush` k-blocks into an FP64 workspace (double-buffered TMEM,
// the flush overlaps the next chunk's MMAs), so FP32 accumulation only spans
// short chunks.
//
// Kernel roles (192 threads): warp 0 issues TMA loads, warp 1 allocates TMEM
// and issues the MMAs, warps 2-5 drain TMEM into the FP64 workspace.  Every
// wait is bounded: on expiry the CTA records an error code and exits.
#include <cuda.h>
#include <cuda_fp16.h>

#include <cstring>
#include <vector>

#include "common.cuh"

namespace isdf {

namespace tc {

constexpr int BM = 128;        // A' rows per tile (64 complex rows of E)
constexpr int BN = 256;        // B' rows per tile (complex columns of E)
constexpr int BK = 64;         // fp16 per row per stage (one 128-byte swizzle row)
constexpr int STAGES = 2;
constexpr int A_BYTES = BM * BK * 2;        // 16 KB
constexpr int B_BYTES = BN * BK * 2;        // 32 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // Ah, Al, Bh, Bl: 96 KB
constexpr int TMEM_COLS = 512;              // two 256-column FP32 accumulators
constexpr int NTHREADS = 192;
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
// Bounded wait for the phase of parity `parity`; false on timeout or if another
// thread of the CTA already gave up.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
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
  double* ws;          // [tile][BN][BM] FP64 partial sums
  int nkb;             // k-blocks of BK
  int flush;           // k-blocks per TMEM chunk
  int* err;            // device error word
};

__global__ void __launch_bounds__(NTHREADS, 1)
    herk_tc_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                   const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, TileArgs args) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment of the shared-window address (128-byte swizzle atoms)
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* full = bars;                 // [STAGES]
  uint64_t* empty = bars + STAGES;       // [STAGES]
  uint64_t* accf = bars + 2 * STAGES;    // [2]
  uint64_t* acce = bars + 2 * STAGES + 2;  // [2]
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
  volatile int* s_err = reinterpret_cast<volatile int*>(s_tmem + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int2 tile = args.tiles[blockIdx.x];
  const int nkb = args.nkb, F = args.flush;
  const int nchunks = (nkb + F - 1) / F;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 128);
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
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % STAGES, r = kb / STAGES;
        if (!mbar_wait(&empty[s], (r & 1) ^ 1, s_err, args.err, 1)) break;
        uint8_t* st = smem + s * STAGE_BYTES;
        mbar_expect_tx(&full[s], STAGE_BYTES);
        const int x = kb * BK;
        tma_load_2d(st, &mAh, &full[s], x, tile.x * BM);
        tma_load_2d(st + A_BYTES, &mAl, &full[s], x, tile.x * BM);
        tma_load_2d(st + 2 * A_BYTES, &mBh, &full[s], x, tile.y * BN);
        tma_load_2d(st + 2 * A_BYTES + B_BYTES, &mBl, &full[s], x, tile.y * BN);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % STAGES, r = kb / STAGES;
        const int c = kb / F, buf = c & 1, u = c >> 1;
        const bool first_in_chunk = (kb % F) == 0;
        if (first_in_chunk) {
          if (!mbar_wait(&acce[buf], (u & 1) ^ 1, s_err, args.err, 2)) break;
          tc_fence_after();
        }
        if (!mbar_wait(&full[s], r & 1, s_err, args.err, 3)) break;
        tc_fence_after();
        const uint8_t* st = smem + s * STAGE_BYTES;
        const uint64_t dAh = sdesc_sw128(st), dAl = sdesc_sw128(st + A_BYTES);
        const uint64_t dBh = sdesc_sw128(st + 2 * A_BYTES), dBl = sdesc_sw128(st + 2 * A_BYTES + B_BYTES);
        const uint32_t d = tmem_base + (uint32_t)(buf * BN);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t off = (uint64_t)(kk * 32) >> 4;  // 16 fp16 = 32 bytes along K
          umma_f16(d, dAh + off, dBh + off, kIdesc, (first_in_chunk && kk == 0) ? 0u : 1u);
          umma_f16(d, dAh + off, dBl + off, kIdesc, 1u);
          umma_f16(d, dAl + off, dBh + off, kIdesc, 1u);
        }
        umma_commit(&empty[s]);
        if ((kb % F) == F - 1 || kb == nkb - 1) umma_commit(&accf[buf]);
      }
    }
  } else {
    // epilogue: warps 2..5 -> TMEM lane quarter (warp % 4)
    const int q = warp & 3;
    const int row = q * 32 + lane;
    double* ws = args.ws + (size_t)blockIdx.x * BN * BM;
    for (int c = 0; c < nchunks; ++c) {
      const int buf = c & 1, u = c >> 1;
      if (!mbar_wait(&accf[buf], u & 1, s_err, args.err, 4)) break;
      tc_fence_after();
#pragma unroll 1
      for (int cb = 0; cb < BN / 32; ++cb) {
        uint32_t v[32];
        tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + cb * 32), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          double* p = ws + (size_t)(cb * 32 + j) * BM + row;
          const double x = (double)__uint_as_float(v[j]);
          if (c == 0)
            *p = x;
          else
            *p += x;
        }
      }
      tc_fence_before();
      mbar_arrive(&acce[buf]);
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
__global__ void maxabs_kernel(const float2* __restrict__ B, int64_t rows, int64_t cols, int64_t ld,
                              unsigned int* __restrict__ out_bits) {
  float m = 0.f;
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = B[(e / cols) * ld + (e % cols)];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out_bits, __float_as_uint(m));  // non-negative floats order as uints
}

// A'[2a][2k] = s Re B_ak, A'[2a][2k+1] = s Im B_ak, A'[2a+1][2k] = s Im B_ak, A'[2a+1][2k+1] = -s Re B_ak,
// split into hi = fp16(x), lo = fp16(x - hi); columns beyond 2K are zero.
__global__ void split_kernel(const float2* __restrict__ B, int64_t n2, int64_t K, int64_t ld, int64_t K2,
                             const unsigned int* __restrict__ maxbits, __half* __restrict__ Ah,
                             __half* __restrict__ Al) {
  const float mx = __uint_as_float(*maxbits);
  // scale: power of two bringing the largest entry to about 2^12
  const float s = mx > 0.f ? exp2f(floorf(12.f - log2f(mx))) : 1.f;
  const int64_t total = n2 * (K2 / 2);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / (K2 / 2), k = e % (K2 / 2);
    float2 v = make_float2(0.f, 0.f);
    if (k < K) v = B[a * ld + k];
    const float pr = s * v.x, pi = s * v.y;
    const float vals[4] = {pr, pi, pi, -pr};
    __half hi[4], lo[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      hi[t] = __float2half_rn(vals[t]);
      lo[t] = __float2half_rn(vals[t] - __half2float(hi[t]));
    }
    const int64_t rP = (2 * a) * K2 + 2 * k, rQ = (2 * a + 1) * K2 + 2 * k;
    *reinterpret_cast<__half2*>(Ah + rP) = __halves2half2(hi[0], hi[1]);
    *reinterpret_cast<__half2*>(Al + rP) = __halves2half2(lo[0], lo[1]);
    *reinterpret_cast<__half2*>(Ah + rQ) = __halves2half2(hi[2], hi[3]);
    *reinterpret_cast<__half2*>(Al + rQ) = __halves2half2(lo[2], lo[3]);
  }
}

// E (complex128, n2 x n2, Hermitian) from the FP64 tile workspace, scaled by
// scale / s^2 where s is the split scale.
__global__ void herk_finish_kernel(const double* __restrict__ ws, const int2* __restrict__ tiles, int ntiles,
                                   int64_t n2, const unsigned int* __restrict__ maxbits, double scale,
                                   double2* __restrict__ E) {
  const float mx = __uint_as_float(*maxbits);
  const double s = mx > 0.f ? (double)exp2f(floorf(12.f - log2f(mx))) : 1.0;
  const double f = scale / (s * s);
  const int64_t per = (int64_t)BN * (BM / 2);
  const int64_t total = per * ntiles;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / per);
    const int c = (int)((e % per) / (BM / 2));
    const int al = (int)(e % (BM / 2));
    const int64_t a = (int64_t)tiles[t].x * (BM / 2) + al;
    const int64_t b = (int64_t)tiles[t].y * BN + c;
    if (a >= n2 || b >= n2 || a < b) continue;
    const double* w = ws + ((size_t)t * BN + c) * BM;
    const double re = w[2 * al] * f, im = w[2 * al + 1] * f;
    E[a * n2 + b] = make_double2(re, im);
    if (a != b) E[b * n2 + a] = make_double2(re, -im);
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
  return (size_t)2 * (2 * n2) * K2 * sizeof(__half);  // hi and lo
}

void herk_tc_tiles(int64_t n2, std::vector<int2>& tiles) {
  tiles.clear();
  const int64_t mt = (2 * n2 + tc::BM - 1) / tc::BM, nt = (n2 + tc::BN - 1) / tc::BN;
  for (int64_t tj = 0; tj < nt; ++tj)
    for (int64_t ti = 0; ti < mt; ++ti)
      if (ti * (tc::BM / 2) + (tc::BM / 2 - 1) >= tj * tc::BN) tiles.push_back(make_int2((int)ti, (int)tj));
}

size_t herk_tc_ws_bytes(int64_t ntiles) { return (size_t)ntiles * tc::BN * tc::BM * sizeof(double); }

// E (complex128 n2 x n2) = scale * B B^H, B complex64 n2 x K (row pitch ldb).
// split: device buffer of herk_tc_split_bytes; tiles_d: device copy of herk_tc_tiles;
// ws: herk_tc_ws_bytes; scratch_u32: 1 device word; err: 1 device int (0 on entry).
cudaError_t herk_tc(cudaStream_t st, const float2* B, int64_t n2, int64_t K, int64_t ldb, double scale,
                    void* split, const int2* tiles_d, int ntiles, double* ws, unsigned int* scratch_u32, int* err,
                    double2* E, int flush) {
  using namespace tc;
  if (n2 <= 0 || K <= 0 || ntiles <= 0) return cudaSuccess;
  const int64_t K2 = ((2 * K + BK - 1) / BK) * BK;
  __half* Ah = reinterpret_cast<__half*>(split);
  __half* Al = Ah + (size_t)(2 * n2) * K2;
  cudaError_t e = cudaMemsetAsync(scratch_u32, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  maxabs_kernel<<<nblk(n2 * K), 256, 0, st>>>(B, n2, K, ldb, scratch_u32);
  count_launch();
  split_kernel<<<nblk(n2 * (K2 / 2)), 256, 0, st>>>(B, n2, K, ldb, K2, scratch_u32, Ah, Al);
  count_launch();
  CUtensorMap mAh, mAl, mBh, mBl;
  if (!make_map(&mAh, Ah, K2, 2 * n2, K2, BM) || !make_map(&mAl, Al, K2, 2 * n2, K2, BM) ||
      !make_map(&mBh, Ah, K2, n2, 2 * K2, BN) || !make_map(&mBl, Al, K2, n2, 2 * K2, BN))
    return cudaErrorInvalidValue;
  const size_t smem = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
  e = cudaFuncSetAttribute(herk_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  TileArgs args{tiles_d, ws, (int)(K2 / BK), flush < 1 ? 1 : flush, err};
  herk_tc_kernel<<<ntiles, NTHREADS, smem, st>>>(mAh, mAl, mBh, mBl, args);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  herk_finish_kernel<<<nblk((int64_t)ntiles * BN * (BM / 2)), 256, 0, st>>>(ws, tiles_d, ntiles, n2, scratch_u32,
                                                                            scale, E);
  count_launch();
  return cudaGetLastError();
}

}  // namespace isdf
