// Batched FP64 factorisations for the least-squares solve (Eq. 3).
//
// pchol_batched  pivoted Cholesky of Hermitian PSD matrices, one block per
//                matrix: pivot = largest remaining diagonal, where diagonals
//                within 1e-11 * (largest initial diagonal) of it are ties
//                resolved to the smallest index; stop when it is <= tol *
//                largest initial diagonal.  Column j of L is stored as Lt[j][:].
// trinv_batched  W = L_S^{-1} for the kept rows S = perm[:rank] (L_S is lower
//                triangular in pivot order), scattered to Wfull[i][perm[c]] so
//                that xi = Wfull * eta and zeta = Wfull^H * xi give the basic
//                least-squares solution (zeta = 0 on dropped points).
#include "common.cuh"

namespace isdf {

namespace {

constexpr double kTieEps = 1e-11;  // pivot tie window, relative to the largest initial diagonal

__global__ void __launch_bounds__(512) pchol_kernel(const double2* __restrict__ A, int n, double tol,
                                                    double2* __restrict__ Lt, int32_t* __restrict__ perm,
                                                    int32_t* __restrict__ rank, double* __restrict__ dwork) {
  const int b = blockIdx.x;
  A += (int64_t)b * n * n;
  Lt += (int64_t)b * n * n;
  perm += (int64_t)b * n;
  double* d = dwork + (int64_t)b * 2 * n;
  double* used = d + n;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_p;
  __shared__ double s_dp;
  __shared__ double s_d0;
  for (int i = tid; i < n; i += blockDim.x) {
    d[i] = A[(int64_t)i * n + i].x;
    used[i] = 0.0;
  }
  __syncthreads();
  int r = 0;
  for (int j = 0; j < n; ++j) {
    // largest remaining diagonal over unused rows
    double bv = -INFINITY;
    for (int i = tid; i < n; i += blockDim.x)
      if (used[i] == 0.0) bv = fmax(bv, d[i]);
    for (int o = 16; o; o >>= 1) bv = fmax(bv, __shfl_xor_sync(0xffffffffu, bv, o));
    if (lane == 0) sv[w] = bv;
    __syncthreads();
    if (tid == 0) {
      double v = sv[0];
      for (int t = 1; t < nw; ++t) v = fmax(v, sv[t]);
      if (j == 0) s_d0 = v;
      s_dp = v;
    }
    __syncthreads();
    const double dmax = s_dp;
    if (!(dmax > tol * s_d0) || !(dmax > 0.0)) break;
    // ties: every unused row within tie_eps * d_max,0 (and >= dmax/2) -> smallest index
    const double thr = fmax(dmax - kTieEps * s_d0, 0.5 * dmax);
    int bi = n;
    for (int i = tid; i < n; i += blockDim.x)
      if (used[i] == 0.0 && d[i] >= thr && i < bi) bi = i;
    for (int o = 16; o; o >>= 1) bi = min(bi, __shfl_xor_sync(0xffffffffu, bi, o));
    if (lane == 0) si[w] = bi;
    __syncthreads();
    if (tid == 0) {
      int ii = si[0];
      for (int t = 1; t < nw; ++t) ii = min(ii, si[t]);
      s_p = ii;
      s_dp = ii < n ? d[ii] : 0.0;
    }
    __syncthreads();
    const int p = s_p;
    if (p >= n) break;  // no finite candidate
    const double dp = s_dp;
    const double inv = 1.0 / sqrt(dp);
    for (int i = tid; i < n; i += blockDim.x) {
      double2 acc = A[(int64_t)i * n + p];
      for (int l = 0; l < j; ++l) {
        const double2 a = Lt[(int64_t)l * n + i];
        const double2 bp = Lt[(int64_t)l * n + p];
        // acc -= a * conj(bp)
        acc.x -= a.x * bp.x + a.y * bp.y;
        acc.y -= a.y * bp.x - a.x * bp.y;
      }
      const double2 col = make_double2(acc.x * inv, acc.y * inv);
      // write after all threads have read Lt[l][p] for l < j (row j is new)
      Lt[(int64_t)j * n + i] = col;
      d[i] -= col.x * col.x + col.y * col.y;
    }
    if (tid == 0) {
      used[p] = 1.0;
      perm[j] = p;
    }
    r = j + 1;
    __syncthreads();
  }
  if (tid == 0) rank[b] = r;
  // zero the unused columns so that consumers can read a full n x n array
  for (int64_t e = (int64_t)r * n + tid; e < (int64_t)n * n; e += blockDim.x) Lt[e] = make_double2(0.0, 0.0);
  for (int i = r + tid; i < n; i += blockDim.x) perm[i] = -1;
}

// work[b][i][c] = (L_S^{-1})[i][c]; thread per column c, forward substitution over i.
__global__ void __launch_bounds__(256) trinv_kernel(const double2* __restrict__ Lt,
                                                    const int32_t* __restrict__ perm,
                                                    const int32_t* __restrict__ rank, int n,
                                                    double2* __restrict__ work) {
  const int b = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  Lt += (int64_t)b * n * n;
  perm += (int64_t)b * n;
  work += (int64_t)b * n * n;
  const int r = rank[b];
  if (c >= r) return;
  // L_S[i][l] = Lt[l][perm[i]]
  for (int i = 0; i < r; ++i) {
    if (i < c) {
      work[(int64_t)i * n + c] = make_double2(0.0, 0.0);
      continue;
    }
    const int pi = perm[i];
    double2 acc = make_double2(i == c ? 1.0 : 0.0, 0.0);
    for (int l = c; l < i; ++l) {
      const double2 Lil = Lt[(int64_t)l * n + pi];
      const double2 wl = work[(int64_t)l * n + c];
      acc.x -= Lil.x * wl.x - Lil.y * wl.y;
      acc.y -= Lil.x * wl.y + Lil.y * wl.x;
    }
    const double2 Lii = Lt[(int64_t)i * n + pi];
    // acc / Lii
    const double den = Lii.x * Lii.x + Lii.y * Lii.y;
    work[(int64_t)i * n + c] =
        make_double2((acc.x * Lii.x + acc.y * Lii.y) / den, (acc.y * Lii.x - acc.x * Lii.y) / den);
  }
}

__global__ void scatter_w_kernel(const double2* __restrict__ work, const int32_t* __restrict__ perm,
                                 const int32_t* __restrict__ rank, int n, int batch,
                                 double2* __restrict__ W) {
  const int64_t total = (int64_t)batch * n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / ((int64_t)n * n));
    const int i = (int)((e / n) % n);
    const int c = (int)(e % n);
    const int r = rank[b];
    if (i < r && c < r) {
      const int col = perm[(int64_t)b * n + c];
      W[(int64_t)b * n * n + (int64_t)i * n + col] = work[e];
    }
  }
}

__global__ void lt_to_row_kernel(const double2* __restrict__ Lt, const int32_t* __restrict__ rank,
                                 int n, int batch, double2* __restrict__ L) {
  const int64_t total = (int64_t)batch * n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / ((int64_t)n * n));
    const int i = (int)((e / n) % n);
    const int j = (int)(e % n);
    L[e] = (j < rank[b]) ? Lt[(int64_t)b * n * n + (int64_t)j * n + i] : make_double2(0.0, 0.0);
  }
}

inline int nblocks(int64_t total) {
  int64_t nb = (total + 255) / 256;
  if (nb > 152 * 32) nb = 152 * 32;
  return nb < 1 ? 1 : (int)nb;
}

}  // namespace

cudaError_t pchol_batched(cudaStream_t st, const double2* A, int n, int batch, double tol, double2* Lt,
                          int32_t* perm, int32_t* rank, double* dwork) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  pchol_kernel<<<batch, 512, 0, st>>>(A, n, tol, Lt, perm, rank, dwork);
  count_launch();
  return cudaGetLastError();
}

cudaError_t trinv_batched(cudaStream_t st, const double2* Lt, const int32_t* perm, const int32_t* rank,
                          int n, int batch, double2* W, double2* work) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  dim3 g((n + 255) / 256, batch);
  // work holds L_S^{-1} in pivot order (lower triangular); entries outside the
  // rank stay zero
  cudaError_t e = cudaMemsetAsync(work, 0, sizeof(double2) * (size_t)batch * n * n, st);
  if (e != cudaSuccess) return e;
  trinv_kernel<<<g, 256, 0, st>>>(Lt, perm, rank, n, work);
  count_launch();
  e = cudaMemsetAsync(W, 0, sizeof(double2) * (size_t)batch * n * n, st);
  if (e != cudaSuccess) return e;
  scatter_w_kernel<<<nblocks((int64_t)batch * n * n), 256, 0, st>>>(work, perm, rank, n, batch, W);
  count_launch();
  return cudaGetLastError();
}

cudaError_t lt_to_rowmajor(cudaStream_t st, const double2* Lt, const int32_t* rank, int n, int batch,
                           double2* L) {
  lt_to_row_kernel<<<nblocks((int64_t)batch * n * n), 256, 0, st>>>(Lt, rank, n, batch, L);
  count_launch();
  return cudaGetLastError();
}

}  // namespace isdf
