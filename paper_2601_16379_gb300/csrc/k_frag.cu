// Fragment-ERI epilogues: the chemist's-order permutation of E and the
// Coulomb / exchange energy traces, plus precision conversions.
//
// With E_{(pq),(rs)} = sum_q [M^q V^q M^q^H]_{(pq),(rs)} (scaled by 1/Nk),
// (pq|rs) = E_{(pq),(sr)}   (Eqs. 19-20 in complex form), and
//   E_J =  1/2 sum gamma_pq gamma_rs (pq|rs),
//   E_K = -1/4 sum gamma_ps gamma_rq (pq|rs)   (closed shell, spin-summed gamma).
// The traces are reduced in FP64 with a fixed order (per-row partials, then a
// single-block sum), so repeated calls give identical bits.
#include <mutex>

#include "../../include/isdf.h"
#include "common.cuh"

namespace isdf {

namespace {

template <typename T, typename TO = T>
__global__ void eri_permute_kernel(const T* __restrict__ E, int nf, double scale, TO* __restrict__ eri) {
  const int64_t n2 = (int64_t)nf * nf;
  const int64_t total = n2 * n2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e % nf);
    const int r = (int)((e / nf) % nf);
    const int64_t pq = e / n2;
    const T v = E[pq * n2 + (int64_t)s * nf + r];
    TO o;
    o.x = v.x * scale;
    o.y = v.y * scale;
    eri[e] = o;
  }
}

// One block per (p q) row: partial J and K sums over (r, s).  kChemist selects
// the input layout: false reads E[(pq)][(sr)], true reads eri[p][q][r][s].
template <typename T, bool kChemist = false>
__global__ void __launch_bounds__(256) traces_rows_kernel(const T* __restrict__ E, int nf,
                                                          const double2* __restrict__ g,
                                                          double2* __restrict__ part) {
  const int64_t n2 = (int64_t)nf * nf;
  const int64_t pq = blockIdx.x;
  const int p = (int)(pq / nf), q = (int)(pq % nf);
  double2 aj = make_double2(0, 0), ak = make_double2(0, 0);
  for (int64_t sr = threadIdx.x; sr < n2; sr += blockDim.x) {
    // consecutive threads take consecutive elements of the row in either layout:
    // E[(pq)][(sr)] (s slow, r fast) or eri[p][q][r][s] (r slow, s fast)
    const int s = kChemist ? (int)(sr % nf) : (int)(sr / nf);
    const int r = kChemist ? (int)(sr / nf) : (int)(sr % nf);
    const T ev = E[pq * n2 + sr];  // = (pq|rs)
    const double2 e2 = make_double2((double)ev.x, (double)ev.y);
    // J: gamma_rs * (pq|rs)
    const double2 grs = g[(int64_t)r * nf + s];
    cfma(aj, grs, e2);
    // K: gamma_ps gamma_rq (pq|rs)
    const double2 t = cmul(g[(int64_t)p * nf + s], g[(int64_t)r * nf + q]);
    cfma(ak, t, e2);
  }
  __shared__ double2 sj[256], sk[256];
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
    // J row contribution multiplied by gamma_pq
    const double2 gpq = g[(int64_t)p * nf + q];
    part[2 * pq] = cmul(gpq, sj[0]);
    part[2 * pq + 1] = sk[0];
  }
}

__global__ void __launch_bounds__(256) traces_final_kernel(const double2* __restrict__ part, int64_t nrows,
                                                           double scale, double* __restrict__ out2) {
  __shared__ double2 sj[256], sk[256];
  double2 aj = make_double2(0, 0), ak = make_double2(0, 0);
  for (int64_t i = threadIdx.x; i < nrows; i += blockDim.x) {
    aj = cadd(aj, part[2 * i]);
    ak = cadd(ak, part[2 * i + 1]);
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
    out2[0] = 0.5 * scale * sj[0].x;
    out2[1] = -0.25 * scale * sk[0].x;
    out2[2] = 0.5 * scale * sj[0].y;
    out2[3] = -0.25 * scale * sk[0].y;
  }
}

// out[b][I][J] = a[b][J][I] * c[b][I][J]  (n x n blocks)
__global__ void hadamard_t_kernel(const double2* __restrict__ a, const double2* __restrict__ c, int n, int nb,
                                  double2* __restrict__ out) {
  const int64_t per = (int64_t)n * n, total = per * nb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / per;
    const int I = (int)((e % per) / n), J = (int)(e % n);
    out[e] = cmul(a[b * per + (int64_t)J * n + I], c[e]);
  }
}

// E_ab <- E_ab + conj(E_{s(a) s(b)}) with s((p q)) = (q p).  Each orbit {e, e'}
// of the involution is handled by the thread of its smaller index, so the
// update is in place without races.
__global__ void swapconj_sym_kernel(double2* __restrict__ E, int nf) {
  const int64_t n2 = (int64_t)nf * nf, total = n2 * n2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / n2, b = e % n2;
    const int64_t sa = (a % nf) * nf + a / nf, sb = (b % nf) * nf + b / nf;
    const int64_t e2 = sa * n2 + sb;
    if (e2 < e) continue;
    const double2 x = E[e];
    if (e2 == e) {
      E[e] = make_double2(2.0 * x.x, 0.0);
    } else {
      const double2 y = E[e2];
      E[e] = make_double2(x.x + y.x, x.y - y.y);
      E[e2] = make_double2(y.x + x.x, y.y - x.y);
    }
  }
}

// out[b] = sw[b] * L[b] for blocks of `per` elements, converted to TO.
template <typename TO>
__global__ void scale_blocks_kernel(const double2* __restrict__ L, int64_t per, int nb, const double* __restrict__ sw,
                                    TO* __restrict__ out) {
  const int64_t total = per * nb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const double w = sw[e / per];
    TO o;
    o.x = L[e].x * w;
    o.y = L[e].y * w;
    out[e] = o;
  }
}

// x[dst] = conj(x[src]) (or a plain copy) for blocks of `per` elements, over
// a list of (dst, src) block pairs.
template <typename T, bool kConj>
__global__ void mirror_kernel(T* __restrict__ x, int64_t per, const int2* __restrict__ pairs, int npairs) {
  const int64_t total = per * npairs;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int2 pr = pairs[e / per];
    const int64_t j = e % per;
    T v = x[(int64_t)pr.y * per + j];
    if constexpr (kConj) v.y = -v.y;
    x[(int64_t)pr.x * per + j] = v;
  }
}

// out[I][mu n_ao + nu] = conj(x1[I][mu]) x2[I][nu]  (AO pair rows of one k-pair)
__global__ void ao_pair_kernel(const double2* __restrict__ x1, const double2* __restrict__ x2, int np, int nao,
                               double2* __restrict__ out) {
  const int64_t n2 = (int64_t)nao * nao, total = (int64_t)np * n2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = e / n2;
    const int mu = (int)((e % n2) / nao), nu = (int)(e % nao);
    const double2 a = x1[I * nao + mu], b = x2[I * nao + nu];
    out[e] = make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
  }
}

// out[k][I][j] = y[k][I][c0 + j] exp(sgn tau eps[k][c0 + j]) for j < nc (columns of the
// orbital values at the points weighted by the imaginary-time factors).
__global__ void scale_cols_kernel(const double2* __restrict__ y, int nk, int np, int nmo, int c0, int nc,
                                  const double* __restrict__ eps, double sgn_tau, double2* __restrict__ out) {
  const int64_t total = (int64_t)nk * np * nc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % nc);
    const int64_t kI = e / nc;
    const int k = (int)(kI / np);
    const double w = exp(sgn_tau * eps[(int64_t)k * nmo + c0 + j]);
    const double2 v = y[kI * nmo + c0 + j];
    out[e] = make_double2(v.x * w, v.y * w);
  }
}

// part[Q] = Re sum_IJ t[Q][I][J] chi[-Q][I][J]  (one block per Q, fixed summation order)
__global__ void __launch_bounds__(256) sos_trace_kernel(const double2* __restrict__ t, const double2* __restrict__ chi,
                                                        int n0, int n1, int n2, int np, double* __restrict__ part) {
  const int Q = blockIdx.x;
  const int q0 = Q / (n1 * n2), q1 = (Q / n2) % n1, q2 = Q % n2;
  const int mQ = (((n0 - q0) % n0) * n1 + (n1 - q1) % n1) * n2 + (n2 - q2) % n2;
  const int64_t pp = (int64_t)np * np;
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < pp; e += blockDim.x) {
    const double2 a = t[(int64_t)Q * pp + e], b = chi[(int64_t)mQ * pp + e];
    acc += a.x * b.x - a.y * b.y;
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[Q] = sh[0];
}

__global__ void z2c_kernel(const double2* __restrict__ in, float2* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = make_float2((float)in[e].x, (float)in[e].y);
}
__global__ void c2z_kernel(const float2* __restrict__ in, double2* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = make_double2((double)in[e].x, (double)in[e].y);
}

inline int nblocks(int64_t total) {
  int64_t nb = (total + 255) / 256;
  if (nb > 152 * 32) nb = 152 * 32;
  return nb < 1 ? 1 : (int)nb;
}

}  // namespace

cudaError_t eri_permute(cudaStream_t st, const double2* E, int nf, double scale, double2* eri) {
  eri_permute_kernel<double2><<<nblocks((int64_t)nf * nf * nf * nf), 256, 0, st>>>(E, nf, scale, eri);
  count_launch();
  return cudaGetLastError();
}
cudaError_t eri_permute_zc(cudaStream_t st, const double2* E, int nf, double scale, float2* eri) {
  eri_permute_kernel<double2, float2><<<nblocks((int64_t)nf * nf * nf * nf), 256, 0, st>>>(E, nf, scale, eri);
  count_launch();
  return cudaGetLastError();
}

// out receives 4 doubles (E_J, E_K and their imaginary parts); part is 2*nf*nf double2
// of scratch.
template <typename T>
static cudaError_t traces_impl(cudaStream_t st, const T* E, int nf, double scale, const double2* gamma,
                               double* out, double2* part) {
  const int64_t n2 = (int64_t)nf * nf;
  traces_rows_kernel<T><<<(unsigned)n2, 256, 0, st>>>(E, nf, gamma, part);
  count_launch();
  traces_final_kernel<<<1, 256, 0, st>>>(part, n2, scale, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t eri_traces(cudaStream_t st, const double2* E, int nf, double scale, const double2* gamma,
                       double* out, double2* part) {
  return traces_impl<double2>(st, E, nf, scale, gamma, out, part);
}

cudaError_t eri_swapconj_sym(cudaStream_t st, double2* E, int nf) {
  swapconj_sym_kernel<<<nblocks((int64_t)nf * nf * nf * nf), 256, 0, st>>>(E, nf);
  count_launch();
  return cudaGetLastError();
}
cudaError_t scale_blocks(cudaStream_t st, const double2* L, int64_t per, int nb, const double* sw, double2* out) {
  scale_blocks_kernel<double2><<<nblocks(per * nb), 256, 0, st>>>(L, per, nb, sw, out);
  count_launch();
  return cudaGetLastError();
}
cudaError_t scale_blocks_f(cudaStream_t st, const double2* L, int64_t per, int nb, const double* sw, float2* out) {
  scale_blocks_kernel<float2><<<nblocks(per * nb), 256, 0, st>>>(L, per, nb, sw, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t ao_pairs(cudaStream_t st, const double2* x1, const double2* x2, int np, int nao, double2* out) {
  ao_pair_kernel<<<nblocks((int64_t)np * nao * nao), 256, 0, st>>>(x1, x2, np, nao, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t scale_cols(cudaStream_t st, const double2* y, int nk, int np, int nmo, int c0, int nc, const double* eps,
                       double sgn_tau, double2* out) {
  if ((int64_t)nk * np * nc == 0) return cudaSuccess;
  scale_cols_kernel<<<nblocks((int64_t)nk * np * nc), 256, 0, st>>>(y, nk, np, nmo, c0, nc, eps, sgn_tau, out);
  count_launch();
  return cudaGetLastError();
}
cudaError_t sos_trace_parts(cudaStream_t st, const double2* t, const double2* chi, const int kmesh[3], int np,
                            double* part) {
  const int nk = kmesh[0] * kmesh[1] * kmesh[2];
  sos_trace_kernel<<<nk, 256, 0, st>>>(t, chi, kmesh[0], kmesh[1], kmesh[2], np, part);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mirror_conj(cudaStream_t st, double2* x, int64_t per, const int2* pairs, int npairs) {
  if (npairs <= 0 || per <= 0) return cudaSuccess;
  mirror_kernel<double2, true><<<nblocks(per * npairs), 256, 0, st>>>(x, per, pairs, npairs);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mirror_copy(cudaStream_t st, int32_t* x, int64_t per, const int2* pairs, int npairs) {
  if (npairs <= 0 || per <= 0) return cudaSuccess;
  mirror_kernel<int32_t, false><<<nblocks(per * npairs), 256, 0, st>>>(x, per, pairs, npairs);
  count_launch();
  return cudaGetLastError();
}

cudaError_t hadamard_t(cudaStream_t st, const double2* a, const double2* c, int n, int nb, double2* out) {
  hadamard_t_kernel<<<nblocks((int64_t)n * n * nb), 256, 0, st>>>(a, c, n, nb, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t z2c(cudaStream_t st, const double2* in, float2* out, int64_t n) {
  z2c_kernel<<<nblocks(n), 256, 0, st>>>(in, out, n);
  count_launch();
  return cudaGetLastError();
}
cudaError_t c2z(cudaStream_t st, const float2* in, double2* out, int64_t n) {
  c2z_kernel<<<nblocks(n), 256, 0, st>>>(in, out, n);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free trace entry point.  Its scratch (per-row partial sums and the
// four result words) lives in a file-scope device array that every GPU loading
// the library holds until the process exits; the host needs the array's device
// address, obtained once per device with cudaGetSymbolAddress.
namespace {
constexpr int64_t kNoAllocScratchDoubles = int64_t(1) << 20;  // 8 MiB: 4 + 4*n_f^2 doubles, n_f <= 511
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};
thread_local char g_noalloc_msg[256] = "";

int noalloc_fail(int code, const char* msg) {
  snprintf(g_noalloc_msg, sizeof(g_noalloc_msg), "%s", msg);
  return code;
}
}  // namespace

const char* noalloc_last_error() { return g_noalloc_msg; }

}  // namespace isdf

extern "C" int isdf_eri_traces_noalloc(const void* eri, int n_orb, const void* gamma, double* ej_out,
                                       double* ek_out, void* cuda_stream) {
  using namespace isdf;
  if (!eri || !gamma || !ej_out || !ek_out || n_orb < 1)
    return noalloc_fail(ISDF_ERR_ARG, "isdf_eri_traces_noalloc: NULL pointer or n_orb < 1");
  const int64_t n2 = (int64_t)n_orb * n_orb;
  if (4 + 4 * n2 > kNoAllocScratchDoubles)
    return noalloc_fail(ISDF_ERR_ARG, "isdf_eri_traces_noalloc: n_orb exceeds the 511-orbital scratch limit");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(ISDF_ERR_CUDA, "isdf_eri_traces_noalloc: no current CUDA device");
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return noalloc_fail(ISDF_ERR_CUDA, "isdf_eri_traces_noalloc: cudaGetSymbolAddress of the scratch failed");
      }
      g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double* out = scratch;                                        // 4 result words
  double2* part = reinterpret_cast<double2*>(scratch + 4);     // 2 * n2 partial sums
  traces_rows_kernel<double2, true><<<(unsigned)n2, 256, 0, st>>>(static_cast<const double2*>(eri), n_orb,
                                                                  static_cast<const double2*>(gamma), part);
  traces_final_kernel<<<1, 256, 0, st>>>(part, n2, 1.0, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(ISDF_ERR_CUDA, cudaGetErrorString(e));
  double hv[2];
  e = cudaMemcpyAsync(hv, out, sizeof(hv), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return noalloc_fail(ISDF_ERR_CUDA, cudaGetErrorString(e));
  *ej_out = hv[0];
  *ek_out = hv[1];
  g_noalloc_msg[0] = '\0';
  return ISDF_OK;
}
