// Batched complex GEMM on the SIMT pipes (FP64 and FP32).
//
// C_b = alpha * op(A_b) * op(B_b) + beta * C_b, row-major, op in {N, T, C, R}.
// Used for the small-K contractions of the fit (G^k = X^k^* X^k^T, g^k = X^k^* Phi^k,
// T^k = X^k C^k), the explicit-factor products of the solve, and the FP64 path's
// Coulomb and fragment contractions (Eqs. 4-6, 19-20).
//
// Tiling: 64 x 64 output tile per 256-thread block, each thread owns a 4 x 4
// sub-tile spread with stride 16 (conflict-free shared reads), K staged 8 (FP64)
// or 16 (FP32) at a time through shared memory.
//
// FP32 accumulation is compensated: each K tile is summed in FP32, then folded
// into a float-float running sum with TwoSum (Knuth), so the rounding error is
// that of a 16-term FP32 sum plus ~2^-48 of the total instead of growing with K.
#include "common.cuh"

namespace isdf {

template <typename T>
struct Scalar;
template <>
struct Scalar<double2> {
  using real = double;
};
template <>
struct Scalar<float2> {
  using real = float;
};

template <typename T>
__device__ __forceinline__ T zero_c() {
  T z;
  z.x = 0;
  z.y = 0;
  return z;
}
template <typename T>
__device__ __forceinline__ T conj_if(T v, bool c) {
  if (c) v.y = -v.y;
  return v;
}
__device__ __forceinline__ void cfma_t(double2& acc, double2 a, double2 b) { cfma(acc, a, b); }
__device__ __forceinline__ void cfma_t(float2& acc, float2 a, float2 b) { cfma(acc, a, b); }

// hi + lo += x, error-free (TwoSum).
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float ap = s - bp;
  lo += (hi - ap) + (x - bp);
  hi = s;
}
__device__ __forceinline__ void fold(double2& acc, double2& lo, double2 part) {
  acc.x += part.x;
  acc.y += part.y;
}
__device__ __forceinline__ void fold(float2& acc, float2& lo, float2 part) {
  two_sum_acc(acc.x, lo.x, part.x);
  two_sum_acc(acc.y, lo.y, part.y);
}
template <typename T>
__device__ __forceinline__ T finish(T acc, T lo);
template <>
__device__ __forceinline__ double2 finish(double2 acc, double2) { return acc; }
template <>
__device__ __forceinline__ float2 finish(float2 acc, float2 lo) {
  return make_float2(acc.x + lo.x, acc.y + lo.y);
}

// Optional structure: lowerA skips the k > row part of a lower-triangular
// op(A); brow (with batch stride sIdx) gathers the rows of B ('N' only):
// op(B)[kk][n] = B[brow[kk]][n], 0 where brow[kk] < 0.
template <typename T, int BK>
__global__ void __launch_bounds__(256, 2) gemm_kernel(char opA, char opB, int m, int n, int k, T alpha,
                                                   const T* __restrict__ A, int64_t lda, int64_t sA,
                                                   const T* __restrict__ B, int64_t ldb, int64_t sB,
                                                   T beta, T* __restrict__ C, int64_t ldc,
                                                   int64_t sC, int lowerA, const int32_t* __restrict__ brow,
                                                   int64_t sIdx) {
  constexpr int BM = 64, BN = 64;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int64_t b = blockIdx.z;
  A += b * sA;
  B += b * sB;
  C += b * sC;
  if (brow) brow += b * sIdx;
  const int kend = lowerA ? min(k, m0 + BM) : k;
  const bool aT = (opA == 'T' || opA == 'C');
  const bool aC = (opA == 'C' || opA == 'R');
  const bool bT = (opB == 'T' || opB == 'C');
  const bool bC = (opB == 'C' || opB == 'R');

  constexpr bool kComp = sizeof(T) == 8;  // compensated accumulation for FP32
  T acc[4][4], lo[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[i][j] = zero_c<T>();
      lo[i][j] = zero_c<T>();
    }

  // Global -> register staging of one K-tile (op(A): BM x BK, op(B): BK x BN), so
  // that the loads of tile k0 + BK are in flight while tile k0 is computed.
  constexpr int NA = (BM * BK) / 256, NB = (BN * BK) / 256;
  T ra[NA], rb[NB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const int e = tid + u * 256;
      int mm, kk;
      if (aT) {
        kk = e / BM;
        mm = e % BM;
      } else {
        mm = e / BK;
        kk = e % BK;
      }
      const int gm = m0 + mm, gk = k0 + kk;
      T v = zero_c<T>();
      if (gm < m && gk < k) v = aT ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
      ra[u] = conj_if(v, aC);
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int e = tid + u * 256;
      int nn, kk;
      if (bT) {
        nn = e / BK;
        kk = e % BK;
      } else {
        kk = e / BN;
        nn = e % BN;
      }
      const int gn = n0 + nn, gk = k0 + kk;
      T v = zero_c<T>();
      if (gn < n && gk < k) {
        if (brow) {
          const int rr = brow[gk];
          if (rr >= 0) v = B[(int64_t)rr * ldb + gn];
        } else {
          v = bT ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn];
        }
      }
      rb[u] = conj_if(v, bC);
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const int e = tid + u * 256;
      if (aT)
        As[e / BM][e % BM] = ra[u];
      else
        As[e % BK][e / BK] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int e = tid + u * 256;
      if (bT)
        Bs[e % BK][e / BK] = rb[u];
      else
        Bs[e / BN][e % BN] = rb[u];
    }
  };
  if (kend > 0) fetch(0);
  for (int k0 = 0; k0 < kend; k0 += BK) {
    stash();
    if (k0 + BK < kend) fetch(k0 + BK);
    __syncthreads();
    if constexpr (kComp) {
      T part[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[i][j] = zero_c<T>();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) cfma_t(part[i][j], a[i], bb[j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) fold(acc[i][j], lo[i][j], part[i][j]);
    } else {
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) cfma_t(acc[i][j], a[i], bb[j]);
      }
    }
    __syncthreads();
  }
  const bool use_beta = (beta.x != 0 || beta.y != 0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= n) continue;
      T r = cmul(alpha, finish(acc[i][j], lo[i][j]));
      T* cp = C + (int64_t)gm * ldc + gn;
      if (use_beta) {
        T o = *cp;
        T t = cmul(beta, o);
        r.x += t.x;
        r.y += t.y;
      }
      *cp = r;
    }
  }
}

template <typename T, int BK>
static cudaError_t gemm_launch(cudaStream_t st, char opA, char opB, int m, int n, int k, T alpha,
                               const T* A, int64_t lda, int64_t sA, const T* B, int64_t ldb,
                               int64_t sB, T beta, T* C, int64_t ldc, int64_t sC, int batch,
                               int lowerA = 0, const int32_t* brow = nullptr, int64_t sIdx = 0) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) {
    // split very large batches
    for (int b0 = 0; b0 < batch; b0 += 65535) {
      int nb = batch - b0 < 65535 ? batch - b0 : 65535;
      cudaError_t e = gemm_launch<T, BK>(st, opA, opB, m, n, k, alpha, A + b0 * sA, lda, sA,
                                         B + b0 * sB, ldb, sB, beta, C + b0 * sC, ldc, sC, nb, lowerA,
                                         brow ? brow + b0 * sIdx : nullptr, sIdx);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  dim3 grid((n + 63) / 64, (m + 63) / 64, batch);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  if (brow && opB != 'N') return cudaErrorInvalidValue;
  gemm_kernel<T, BK><<<grid, 256, 0, st>>>(opA, opB, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta,
                                           C, ldc, sC, lowerA, brow, sIdx);
  count_launch();
  return cudaGetLastError();
}

cudaError_t zgemm(cudaStream_t st, char opA, char opB, int m, int n, int k, double2 alpha,
                  const double2* A, int64_t lda, int64_t sA, const double2* B, int64_t ldb,
                  int64_t sB, double2 beta, double2* C, int64_t ldc, int64_t sC, int batch) {
  return gemm_launch<double2, 8>(st, opA, opB, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C,
                                 ldc, sC, batch);
}

cudaError_t ztrmm_gather(cudaStream_t st, int m, int n, const double2* A, int64_t lda, int64_t sA,
                         const int32_t* brow, int64_t sIdx, const double2* B, int64_t ldb, int64_t sB, double2* C,
                         int64_t ldc, int64_t sC, int batch) {
  return gemm_launch<double2, 8>(st, 'N', 'N', m, n, m, make_double2(1.0, 0.0), A, lda, sA, B, ldb, sB,
                                 make_double2(0.0, 0.0), C, ldc, sC, batch, 1, brow, sIdx);
}

cudaError_t cgemm(cudaStream_t st, char opA, char opB, int m, int n, int k, float2 alpha,
                  const float2* A, int64_t lda, int64_t sA, const float2* B, int64_t ldb,
                  int64_t sB, float2 beta, float2* C, int64_t ldc, int64_t sC, int batch) {
  return gemm_launch<float2, 16>(st, opA, opB, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C,
                                 ldc, sC, batch);
}

}  // namespace isdf
