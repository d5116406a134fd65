// FP64-accurate complex GEMM on the tensor cores for a short inner dimension:
//     C_b[i][j] = sum_m op(A_b)[i][m] B_b[m][j],   op(A) = A ('N') or conj(A) ('R'),
// A_b: M x K, B_b: K x N, C_b: M x N, complex128 row-major, 2K <= 128.  It forms
// g^k = conj(X^k) Phi^k of the fit (Eq. 5), whose inner dimension is N_AO.
//
// Error-free slicing after Ozaki, Ogita, Oishi & Rump (2012).  Real rows
//     A': P_i = (Re a_i1, Im a_i1, Re a_i2, ...),  Q_i = (Im a_i1, -Re a_i1, ...)   (a = op(A))
//     B': R_j = (Re b_1j, -Im b_1j, Re b_2j, -Im b_2j, ...)
// give (A' B'^T)[P_i][j] = Re c_ij and (A' B'^T)[Q_i][j] = Im c_ij.  Each row of A'
// and of B' is scaled by a power of two so that its largest entry lies in
// [64, 128) and written as seven integer slices of 7 bits,
//     v = s1 + s2/2^7 + ... + s7/2^42 (+ remainder below 2^-43),  |s1| <= 128, |s_>1| <= 64,
// stored as fp16 (exact).  The 28 fp16 products S_a T_b with a + b <= 8 feed seven
// FP32 TMEM accumulators by weight 2^{-7(a+b-2)}.  With 2K <= 128 every partial sum
// of a group is an integer of magnitude at most 7 * 2^14 * 128 < 2^24, so the
// accumulation is exact whatever its rounding; the epilogue sums the groups in
// FP64 and rescales.  The dropped products and the slicing remainder leave an
// error of ~2^-48 of |a_i| |b_j| (the rows' largest entries).
//
// Kernel roles (192 threads): warp 0 loads the 14 slice tiles of a k-block by
// TMA, warp 1 allocates TMEM and issues the MMAs, warps 2-5 combine the groups
// and store C.  Every wait is bounded.
#include "common.cuh"
#include "tc_ptx.cuh"

namespace isdf {

namespace {

using namespace tc;

constexpr int ESL = 7;              // slices per operand
constexpr int EBM = 128;            // A' rows per tile (64 complex rows of C)
constexpr int EBN = 64;             // B' rows per tile (complex columns of C)
constexpr int EBK = 64;             // fp16 per row and k-block (one 128-byte swizzle row)
constexpr int EA_BYTES = EBM * EBK * 2;             // 16 KB
constexpr int EB_BYTES = EBN * EBK * 2;             // 8 KB
constexpr int ESTAGE = ESL * (EA_BYTES + EB_BYTES);  // 168 KB
constexpr int ETMEM = 512;                           // 7 groups x 64 columns
constexpr int ENT = 192;
constexpr uint32_t kIdescE = (1u << 4) | ((uint32_t)(EBN >> 3) << 17) | ((uint32_t)(EBM >> 4) << 24);

struct EmuArgs {
  double2* C;
  int64_t ldc, sC;
  int M, N, nkb;
  int mpad2, npad;            // padded rows of A' and B' per batch entry
  const int* rexpA;           // [b][mpad2]
  const int* rexpB;           // [b][npad]
  int* err;
};

__global__ void __launch_bounds__(ENT, 1)
    zgemm_emu_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB, EmuArgs args) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  // one single-use barrier pair per k-block (at most 2): landed, consumed by the MMAs
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + ESTAGE);
  uint64_t* full = bars;       // [2]
  uint64_t* used = bars + 2;   // [2]
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 4);
  volatile int* s_err = reinterpret_cast<volatile int*>(s_tmem + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = args.mpad2 / EBM;
  const int ti = blockIdx.x % mt, tj = blockIdx.x / mt, b = blockIdx.y;
  const int nkb = args.nkb;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&used[i], 1);
    }
    *s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(ETMEM)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      // one stage, reused: k-block kb waits until the MMAs of kb - 1 have read it
      for (int kb = 0; kb < nkb; ++kb) {
        if (kb > 0 && !mbar_wait(&used[kb - 1], 0, s_err, args.err, 21)) break;
        mbar_expect_tx(&full[kb], ESTAGE);
        const int x = kb * EBK;
        for (int i = 0; i < ESL; ++i) {
          // slice i of A' is the row block (i, b) of a [slice][batch][mpad2] stack, likewise B'
          const int ya = (i * (int)gridDim.y + b) * args.mpad2 + ti * EBM;
          const int yb = (i * (int)gridDim.y + b) * args.npad + tj * EBN;
          tma_load_2d(smem + i * EA_BYTES, &mA, &full[kb], x, ya);
          tma_load_2d(smem + ESL * EA_BYTES + i * EB_BYTES, &mB, &full[kb], x, yb);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        if (!mbar_wait(&full[kb], 0, s_err, args.err, 22)) {
          ok = false;
          break;
        }
        tc_fence_after();
        uint64_t dA[ESL], dB[ESL];
#pragma unroll
        for (int i = 0; i < ESL; ++i) {
          dA[i] = sdesc_sw128(smem + i * EA_BYTES);
          dB[i] = sdesc_sw128(smem + ESL * EA_BYTES + i * EB_BYTES);
        }
#pragma unroll
        for (int kk = 0; kk < EBK / 16; ++kk) {
          const uint64_t off = (uint64_t)(kk * 32) >> 4;
#pragma unroll
          for (int g = 0; g < ESL; ++g)
#pragma unroll
            for (int a = 0; a <= g; ++a) {
              // products S_{a+1} T_{g-a+1} of weight 2^{-7g}; the first of a group starts it
              const uint32_t acc = (kb == 0 && kk == 0 && a == 0) ? 0u : 1u;
              umma_f16(tmem_base + (uint32_t)(g * EBN), dA[a] + off, dB[g - a] + off, kIdescE, acc);
            }
        }
        umma_commit(&used[kb]);
      }
    }
  } else {
    // epilogue: warps 2..5 -> TMEM lane quarter (warp % 4); rows P_i / Q_i are lanes 2i / 2i+1
    const int q = warp & 3;
    const int r = q * 32 + lane;
    const int64_t R = (int64_t)ti * EBM + r;  // row of A'
    const int al = r >> 1, part = r & 1;
    // the commit of the last k-block arrives after all earlier MMAs have completed
    const bool okw = __all_sync(0xffffffffu, mbar_wait(&used[nkb - 1], 0, s_err, args.err, 23));
    tc_fence_after();
    // the operand stage is idle now: stage the 64 x 64 complex128 tile for coalesced stores
    constexpr int kPitch = 2 * EBN + 1;  // doubles per staged row
    double* tileS = reinterpret_cast<double*>(smem);
    const int ea = okw ? args.rexpA[(int64_t)b * args.mpad2 + R] : 0;
    const int* fcol = args.rexpB + (int64_t)b * args.npad + tj * EBN;
#pragma unroll 1
    for (int cb = 0; cb < EBN / 32; ++cb) {
      double acc[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = 0.0;
      if (okw) {
#pragma unroll 1
        for (int g = ESL - 1; g >= 0; --g) {
          uint32_t v[32];
          tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * EBN + cb * 32), v);
          const double w = ldexp(1.0, -7 * g);
#pragma unroll
          for (int j = 0; j < 32; ++j) acc[j] = fma((double)__uint_as_float(v[j]), w, acc[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int jl = cb * 32 + j;
        tileS[al * kPitch + 2 * jl + part] = ldexp(acc[j], -(ea + fcol[jl]));
      }
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (okw) {
      const int t = threadIdx.x - 64;
      double2* Cb = args.C + (int64_t)b * args.sC;
      for (int idx = t; idx < (EBM / 2) * EBN; idx += 128) {
        const int ar = idx / EBN, jl = idx % EBN;
        const int64_t ii = (int64_t)ti * (EBM / 2) + ar;
        const int j = tj * EBN + jl;
        if (ii < args.M && j < args.N)
          Cb[ii * args.ldc + j] = make_double2(tileS[ar * kPitch + 2 * jl], tileS[ar * kPitch + 2 * jl + 1]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(ETMEM) : "memory");
  }
}

// Seven integer slices of v (|v| < 128) as fp16.
__device__ __forceinline__ void slice7(double v, __half (&h)[ESL]) {
#pragma unroll
  for (int t = 0; t < ESL; ++t) {
    const double s = rint(v);
    h[t] = __float2half_rn((float)s);
    v = (v - s) * 128.0;
  }
}

__device__ __forceinline__ int row_exp64(double m) { return (m > 0.0 && isfinite(m)) ? 6 - ilogb(m) : 0; }

// A' slices: one warp per complex row i of op(A_b) (K <= 64 entries): rows P_i, Q_i,
// exponent over both; zero rows and columns up to the padding.
__global__ void aslice_kernel(const double2* __restrict__ A, int64_t lda, int64_t sA, int conj, int M, int K, int Kp,
                              int mpad2, int batch, __half* __restrict__ S, int* __restrict__ rexp) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t rows = (int64_t)batch * (mpad2 / 2);
  if (wid >= rows) return;
  const int b = (int)(wid / (mpad2 / 2)), i = (int)(wid % (mpad2 / 2));
  const double2* a = A + (int64_t)b * sA + (int64_t)i * lda;
  double m = 0.0;
  for (int k = lane; k < K; k += 32)
    if (i < M) m = fmax(m, fmax(fabs(a[k].x), fabs(a[k].y)));
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int ex = row_exp64(m);
  const int64_t rowP = (int64_t)b * mpad2 + 2 * i, plane = (int64_t)batch * mpad2 * Kp;
  if (lane == 0) {
    rexp[rowP] = ex;
    rexp[rowP + 1] = ex;
  }
  for (int k = lane; k < Kp / 2; k += 32) {
    double re = 0.0, im = 0.0;
    if (i < M && k < K) {
      re = ldexp(a[k].x, ex);
      im = ldexp(conj ? -a[k].y : a[k].y, ex);
    }
    __half p0[ESL], p1[ESL], q0[ESL], q1[ESL];
    slice7(re, p0);
    slice7(im, p1);
    slice7(im, q0);
    slice7(-re, q1);
#pragma unroll
    for (int s = 0; s < ESL; ++s) {
      *reinterpret_cast<__half2*>(S + s * plane + rowP * Kp + 2 * k) = __halves2half2(p0[s], p1[s]);
      *reinterpret_cast<__half2*>(S + s * plane + (rowP + 1) * Kp + 2 * k) = __halves2half2(q0[s], q1[s]);
    }
  }
}

// B' slices: one thread per column j of B_b: the row R_j = (Re b_mj, -Im b_mj)_m,
// exponent over it; zero rows and columns up to the padding.
__global__ void bslice_kernel(const double2* __restrict__ B, int64_t ldb, int64_t sB, int N, int K, int Kp, int npad,
                              int batch, __half* __restrict__ S, int* __restrict__ rexp) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)batch * npad) return;
  const int b = (int)(e / npad), j = (int)(e % npad);
  const double2* col = B + (int64_t)b * sB + j;
  double m = 0.0;
  if (j < N)
    for (int k = 0; k < K; ++k) m = fmax(m, fmax(fabs(col[(int64_t)k * ldb].x), fabs(col[(int64_t)k * ldb].y)));
  const int ex = row_exp64(m);
  rexp[e] = ex;
  const int64_t plane = (int64_t)batch * npad * Kp;
  for (int k = 0; k < Kp / 2; ++k) {
    double re = 0.0, im = 0.0;
    if (j < N && k < K) {
      const double2 v = col[(int64_t)k * ldb];
      re = ldexp(v.x, ex);
      im = -ldexp(v.y, ex);
    }
    __half h0[ESL], h1[ESL];
    slice7(re, h0);
    slice7(im, h1);
#pragma unroll
    for (int s = 0; s < ESL; ++s)
      *reinterpret_cast<__half2*>(S + s * plane + e * Kp + 2 * k) = __halves2half2(h0[s], h1[s]);
  }
}

int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

bool zgemm_emu_supported(int K) { return K >= 1 && 2 * K <= 2 * EBK; }

size_t zgemm_emu_work_bytes(int M, int N, int K, int batch) {
  const int64_t Kp = rup(2 * (int64_t)K, EBK), mpad2 = rup(2 * (int64_t)M, EBM), npad = rup(N, EBN);
  return (size_t)ESL * batch * (mpad2 + npad) * Kp * sizeof(__half) + sizeof(int) * batch * (mpad2 + npad) + 1024;
}

cudaError_t zgemm_emu(cudaStream_t st, char opA, int M, int N, int K, const double2* A, int64_t lda, int64_t sA,
                      const double2* B, int64_t ldb, int64_t sB, double2* C, int64_t ldc, int64_t sC, int batch,
                      void* work, int* err) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (!zgemm_emu_supported(K) || (opA != 'N' && opA != 'R') || batch > 65535) return cudaErrorInvalidValue;
  const int Kp = (int)rup(2 * (int64_t)K, EBK), mpad2 = (int)rup(2 * (int64_t)M, EBM), npad = (int)rup(N, EBN);
  const int64_t rowsA = (int64_t)ESL * batch * mpad2, rowsB = (int64_t)ESL * batch * npad;
  if (rowsA > 2147483647LL || rowsB > 2147483647LL) return cudaErrorInvalidValue;
  __half* SA = reinterpret_cast<__half*>(work);
  __half* SB = SA + (size_t)rowsA * Kp;
  int* eA = reinterpret_cast<int*>(SB + (size_t)rowsB * Kp);
  int* eB = eA + (size_t)batch * mpad2;
  {
    const int64_t warps = (int64_t)batch * (mpad2 / 2);
    aslice_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(A, lda, sA, opA == 'R', M, K, Kp, mpad2,
                                                                          batch, SA, eA);
    count_launch();
    const int64_t n = (int64_t)batch * npad;
    bslice_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(B, ldb, sB, N, K, Kp, npad, batch, SB, eB);
    count_launch();
  }
  CUtensorMap mA, mB;
  if (!make_map(&mA, SA, Kp, rowsA, Kp, EBM) || !make_map(&mB, SB, Kp, rowsB, Kp, EBN)) return cudaErrorInvalidValue;
  const size_t smem = (size_t)ESTAGE + 1024 + 256;
  cudaError_t e = cudaFuncSetAttribute(zgemm_emu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  EmuArgs args{C, ldc, sC, M, N, Kp / EBK, mpad2, npad, eA, eB, err};
  zgemm_emu_kernel<<<dim3((mpad2 / EBM) * (npad / EBN), batch), ENT, smem, st>>>(mA, mB, args);
  count_launch();
  return cudaGetLastError();
}

}  // namespace isdf
