// Small DFTs of the k-ISDF path.
//
// kdft_cols      transforms along the k-mesh for many independent columns: the
//                convolution theorem of Algorithm 1 (Pi^q, eta^q: k -> R, |.|^2,
//                R -> q) and Algorithm 2 (T^k -> T^R, pair products, R -> q).
// grid_coulomb   cell-grid FFT of e^{-iq.r} x(r) with the 4 pi/|q+G|^2 weight
//                (Eq. 6), producing sqrt(w) c(G) so that V = Omega c'^H c'.
// pair_products  the outer product of Algorithm 2 in supercell space.
//
// All transforms are direct per-axis DFTs staged through shared memory (mesh
// axes are at most 16 points for the k-mesh and 64 for the grid), with the
// twiddles exp(+-2 pi i j/n) tabulated on the host.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "ff.cuh"

namespace isdf {

namespace {

template <typename T>
struct CT {};
template <>
struct CT<double2> {
  using R = double;
  __device__ static double2 mk(double a, double b) { return make_double2(a, b); }
};
template <>
struct CT<float2> {
  using R = float;
  __device__ static float2 mk(float a, float b) { return make_float2(a, b); }
};
// float-float complex: the FP64-class path's transforms in FP32 arithmetic
template <>
struct CT<ffcomplex> {
  using R = ffloat;
  __device__ static ffcomplex mk(ffloat a, ffloat b) { return ffcomplex{a, b}; }
};

// Storage <-> working type of a transform: the same type, or complex128 data
// transformed in float-float.
template <typename T, typename TS>
struct Cv {
  __device__ static T in(const TS& v) { return v; }
  __device__ static TS out(const T& v) { return v; }
};
template <>
struct Cv<ffcomplex, double2> {
  __device__ static ffcomplex in(const double2& v) { return ffcomplex{ffloat(v.x), ffloat(v.y)}; }
  __device__ static double2 out(const ffcomplex& v) { return make_double2(v.x.to_double(), v.y.to_double()); }
};

struct Twiddles16 {
  double c[3][16];
  double s[3][16];
};

Twiddles16 make_tw(const int n[3], int sign) {
  Twiddles16 t;
  for (int a = 0; a < 3; ++a)
    for (int j = 0; j < 16; ++j) {
      double ang = (n[a] > 0 && j < n[a]) ? 2.0 * M_PI * (double)j / (double)n[a] : 0.0;
      t.c[a][j] = std::cos(ang);
      t.s[a][j] = sign * std::sin(ang);
    }
  return t;
}

// In-place DFT along the three k-mesh axes of s[k][c] (Nk x ct), line per thread.
// tc/ts: twiddle cos/sin tables [3][16] in the working precision (shared memory).
template <typename T>
__device__ void kmesh_dft_smem(T* s, int ct, const int n[3], const typename CT<T>::R* tc,
                               const typename CT<T>::R* ts) {
  using R = typename CT<T>::R;
  const int nk = n[0] * n[1] * n[2];
  for (int a = 2; a >= 0; --a) {
    const int L = n[a];
    if (L == 1) continue;
    const int stride = (a == 2) ? 1 : (a == 1 ? n[2] : n[1] * n[2]);
    const int nlines = (nk / L) * ct;
    for (int line = threadIdx.x; line < nlines; line += blockDim.x) {
      const int c = line % ct;
      const int rest = line / ct;  // index over the other two axes
      // base k index with m_a = 0
      const int hi = rest / stride, lo = rest % stride;
      const int base = hi * stride * L + lo;
      T v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (i < L) v[i] = s[(base + i * stride) * ct + c];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (j >= L) break;
        R ax = 0, ay = 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          if (i >= L) break;
          const int t = (i * j) % L;
          const R cr = tc[a * 16 + t], ci = ts[a * 16 + t];
          ax += v[i].x * cr - v[i].y * ci;
          ay += v[i].x * ci + v[i].y * cr;
        }
        s[(base + j * stride) * ct + c] = CT<T>::mk(ax, ay);
      }
    }
    __syncthreads();
  }
}

// Small DFTs in registers for a compile-time length N, as a sub-transform of
// an L-point table: W_N^t = (wc[(t S) mod L], ws[(t S) mod L]) with S = L / N
// (the table holds exp(+-2 pi i t/L), the sign baked into ws).  Composite N
// goes by Cooley-Tukey over its smallest prime factor P (N = P Q):
//   X[k1 + P k2] = sum_n2 W_N^{n2 k1} W_Q^{n2 k2} sum_n1 x[Q n1 + n2] W_P^{n1 k1};
// N = 2, 3 and 5 are written out with the symmetric pairs (x_j +- x_{N-j})
// so that each output costs a few real multiplies; other primes fall back to
// the direct sum.
constexpr int smallest_factor(int n) {
  for (int f = 2; f * f <= n; ++f)
    if (n % f == 0) return f;
  return n;
}

template <typename R, int N, int S, int L, int P = smallest_factor(N)>
struct Dft {
  __host__ __device__ __forceinline__ static void run(R* xr, R* xi, const R* wc, const R* ws) {
    constexpr int Q = N / P;
    R yr[N], yi[N];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) {
      R ar[P], ai[P];
#pragma unroll
      for (int n1 = 0; n1 < P; ++n1) {
        ar[n1] = xr[Q * n1 + n2];
        ai[n1] = xi[Q * n1 + n2];
      }
      Dft<R, P, S * Q, L>::run(ar, ai, wc, ws);
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) {
        // twiddle W_N^{n2 k1}
        const int t = (n2 * k1 * S) % L;
        if (t == 0) {
          yr[k1 * Q + n2] = ar[k1];
          yi[k1 * Q + n2] = ai[k1];
        } else {
          yr[k1 * Q + n2] = ar[k1] * wc[t] - ai[k1] * ws[t];
          yi[k1 * Q + n2] = ar[k1] * ws[t] + ai[k1] * wc[t];
        }
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      R br[Q], bi[Q];
#pragma unroll
      for (int n2 = 0; n2 < Q; ++n2) {
        br[n2] = yr[k1 * Q + n2];
        bi[n2] = yi[k1 * Q + n2];
      }
      Dft<R, Q, S * P, L>::run(br, bi, wc, ws);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) {
        xr[k1 + P * k2] = br[k2];
        xi[k1 + P * k2] = bi[k2];
      }
    }
  }
};

// prime N without a written-out form: the direct sum
template <typename R, int N, int S, int L>
struct Dft<R, N, S, L, N> {
  __host__ __device__ __forceinline__ static void run(R* xr, R* xi, const R* wc, const R* ws) {
    R or_[N], oi[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      R ax = 0, ay = 0;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int t = ((i * j) % N) * S % L;
        ax += xr[i] * wc[t] - xi[i] * ws[t];
        ay += xr[i] * ws[t] + xi[i] * wc[t];
      }
      or_[j] = ax;
      oi[j] = ay;
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
      xr[j] = or_[j];
      xi[j] = oi[j];
    }
  }
};

template <typename R, int S, int L>
struct Dft<R, 1, S, L, 1> {
  __host__ __device__ __forceinline__ static void run(R*, R*, const R*, const R*) {}
};

template <typename R, int S, int L>
struct Dft<R, 2, S, L, 2> {
  __host__ __device__ __forceinline__ static void run(R* xr, R* xi, const R*, const R*) {
    const R r0 = xr[0], i0 = xi[0];
    xr[0] = r0 + xr[1];
    xi[0] = i0 + xi[1];
    xr[1] = r0 - xr[1];
    xi[1] = i0 - xi[1];
  }
};

// W = W_3^1 = c + i s:  X0 = x0 + a,  X1,2 = x0 + c a +- i s b  with a = x1 + x2, b = x1 - x2
template <typename R, int S, int L>
struct Dft<R, 3, S, L, 3> {
  __host__ __device__ __forceinline__ static void run(R* xr, R* xi, const R* wc, const R* ws) {
    const R c = wc[S % L], s = ws[S % L];
    const R ar = xr[1] + xr[2], ai = xi[1] + xi[2], br = xr[1] - xr[2], bi = xi[1] - xi[2];
    const R tr = xr[0] + c * ar, ti = xi[0] + c * ai;
    xr[0] += ar;
    xi[0] += ai;
    xr[1] = tr - s * bi;
    xi[1] = ti + s * br;
    xr[2] = tr + s * bi;
    xi[2] = ti - s * br;
  }
};

// W = W_5^1 = c1 + i s1, W^2 = c2 + i s2; a_j = x_j + x_{5-j}, b_j = x_j - x_{5-j}:
//   X1,4 = x0 + c1 a1 + c2 a2 +- i (s1 b1 + s2 b2),  X2,3 = x0 + c2 a1 + c1 a2 +- i (s2 b1 - s1 b2)
template <typename R, int S, int L>
struct Dft<R, 5, S, L, 5> {
  __host__ __device__ __forceinline__ static void run(R* xr, R* xi, const R* wc, const R* ws) {
    const R c1 = wc[S % L], s1 = ws[S % L], c2 = wc[(2 * S) % L], s2 = ws[(2 * S) % L];
    const R a1r = xr[1] + xr[4], a1i = xi[1] + xi[4], b1r = xr[1] - xr[4], b1i = xi[1] - xi[4];
    const R a2r = xr[2] + xr[3], a2i = xi[2] + xi[3], b2r = xr[2] - xr[3], b2i = xi[2] - xi[3];
    const R t1r = xr[0] + c1 * a1r + c2 * a2r, t1i = xi[0] + c1 * a1i + c2 * a2i;
    const R t2r = xr[0] + c2 * a1r + c1 * a2r, t2i = xi[0] + c2 * a1i + c1 * a2i;
    const R u1r = s1 * b1r + s2 * b2r, u1i = s1 * b1i + s2 * b2i;  // i u1 = (-u1i, u1r)
    const R u2r = s2 * b1r - s1 * b2r, u2i = s2 * b1i - s1 * b2i;
    xr[0] += a1r + a2r;
    xi[0] += a1i + a2i;
    xr[1] = t1r - u1i;
    xi[1] = t1i + u1r;
    xr[4] = t1r + u1i;
    xi[4] = t1i - u1r;
    xr[2] = t2r - u2i;
    xi[2] = t2i + u2r;
    xr[3] = t2r + u2i;
    xi[3] = t2i - u2r;
  }
};

// Cubic mesh of compile-time side L: the three per-axis passes in place on
// s[k][c] (Nk x ct, ct = 2^lct columns), line per thread, with the mixed-radix
// DFT above in registers.  Element (k, c) sits at (k << lct) + c + (k / L) padk:
// the padding after each group of L rows shifts the lines that one 128-byte
// shared-memory phase serves onto different banks (see kdft_cubic_pad).
template <typename T, int L>
__device__ __forceinline__ int cidx(int k, int c, int lct, int padk) {
  return (k << lct) + c + (k / L) * padk;
}

template <typename T, int L>
__device__ void kmesh_dft_cubic(T* s, int lct, int padk, const typename CT<T>::R* tcs, const typename CT<T>::R* tss) {
  using R = typename CT<T>::R;
  R wc[L], ws[L];
#pragma unroll
  for (int t = 0; t < L; ++t) {
    wc[t] = tcs[t];
    ws[t] = tss[t];
  }
  const int ct = 1 << lct, nlines = L * L * ct;
#pragma unroll
  for (int a = 2; a >= 0; --a) {
    const int stride = (a == 2) ? 1 : (a == 1 ? L : L * L);
    for (int line = threadIdx.x; line < nlines; line += blockDim.x) {
      const int c = line & (ct - 1);
      const int rest = line >> lct;
      const int hi = rest / stride, lo = rest % stride;
      const int base = hi * stride * L + lo;
      R vr[L], vi[L];
#pragma unroll
      for (int i = 0; i < L; ++i) {
        const T v = s[cidx<T, L>(base + i * stride, c, lct, padk)];
        vr[i] = v.x;
        vi[i] = v.y;
      }
      Dft<R, L, 1, L>::run(vr, vi, wc, ws);
#pragma unroll
      for (int j = 0; j < L; ++j) s[cidx<T, L>(base + j * stride, c, lct, padk)] = CT<T>::mk(vr[j], vi[j]);
    }
    __syncthreads();
  }
}

template <typename T, int L, typename TS = T>
__global__ void __launch_bounds__(256) kdft_cubic_kernel(TS* __restrict__ data, int64_t ncol, int lct, int padk,
                                                         int mode, Twiddles16 tw1, Twiddles16 tw2, double scale) {
  using R = typename CT<T>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  __shared__ R tw1c[16], tw1s[16], tw2c[16], tw2s[16];
  for (int t = threadIdx.x; t < 16; t += blockDim.x) {
    tw1c[t] = (R)tw1.c[0][t];
    tw1s[t] = (R)tw1.s[0][t];
    tw2c[t] = (R)tw2.c[0][t];
    tw2s[t] = (R)tw2.s[0][t];
  }
  constexpr int nk = L * L * L;
  const int ct = 1 << lct;
  const int64_t c0 = (int64_t)blockIdx.x << lct;
  for (int e = threadIdx.x; e < nk * ct; e += blockDim.x) {
    const int k = e >> lct, c = e & (ct - 1);
    const int64_t col = c0 + c;
    T v = CT<T>::mk(0, 0);
    if (col < ncol) v = Cv<T, TS>::in(data[(int64_t)k * ncol + col]);
    s[cidx<T, L>(k, c, lct, padk)] = v;
  }
  __syncthreads();
  kmesh_dft_cubic<T, L>(s, lct, padk, tw1c, tw1s);
  if (mode == 1) {
    for (int e = threadIdx.x; e < nk * ct; e += blockDim.x) {
      const int i = cidx<T, L>(e >> lct, e & (ct - 1), lct, padk);
      const T v = s[i];
      s[i] = CT<T>::mk(v.x * v.x + v.y * v.y, 0);
    }
    __syncthreads();
    kmesh_dft_cubic<T, L>(s, lct, padk, tw2c, tw2s);
  }
  for (int e = threadIdx.x; e < nk * ct; e += blockDim.x) {
    const int k = e >> lct, c = e & (ct - 1);
    const int64_t col = c0 + c;
    if (col < ncol) {
      const T v = s[cidx<T, L>(k, c, lct, padk)];
      data[(int64_t)k * ncol + col] = Cv<T, TS>::out(CT<T>::mk(v.x * (R)scale, v.y * (R)scale));
    }
  }
}

// DFT along the k-mesh of real columns, out of place, keeping the q with
// qslot[q] >= 0:  out[qslot[q]][col] = scale sum_k e^{s 2 pi i m_q.m_k/n} in[k][col].
// The real pair rows of the time-reversal basis give M^{-q} = conj(M^q), so
// the half set of q in qslot carries all of it.  Two adjacent real columns x =
// col 2c, y = col 2c + 1 share one complex working column z = x + i y, so a row
// of the shared working array is a plain copy of an input row (loaded as
// 16-byte vectors, eight in flight per thread); after the transform
// X(q) = (Z(q) + conj(Z(-q)))/2 and Y(q) = (Z(q) - conj(Z(-q)))/(2i), written
// side by side.
template <typename T, int L>
__global__ void __launch_bounds__(256) kdft_real_cubic_kernel(const typename CT<T>::R* __restrict__ in,
                                                              T* __restrict__ out, int64_t ncol, int lct, int padk,
                                                              const int* __restrict__ qslot, Twiddles16 tw,
                                                              double scale, int vec) {
  using R = typename CT<T>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  __shared__ R twc[16], tws[16];
  for (int t = threadIdx.x; t < 16; t += blockDim.x) {
    twc[t] = (R)tw.c[0][t];
    tws[t] = (R)tw.s[0][t];
  }
  constexpr int nk = L * L * L;
  const int ct = 1 << lct;
  const int64_t c0 = (int64_t)blockIdx.x << (lct + 1);  // 2 ct real columns per block
  if (vec) {
    // 16-byte vectors: EPV working columns each, copied global -> shared by cp.async so
    // that the whole tile is in flight at once; every vector lies wholly inside or
    // outside [0, ncol) (ncol and c0 are multiples of 2 EPV), and its shared slot
    // (k << lct) + cv EPV + (k / L) padk is a multiple of EPV elements (padk is even
    // when ct is), i.e. 16-byte aligned
    constexpr int EPV = 16 / (int)sizeof(T);
    const int vpr = ct / EPV, total = nk * vpr;
    for (int v = threadIdx.x; v < total; v += blockDim.x) {
      const int k = v / vpr, cv = v % vpr;
      const int64_t col = c0 + 2 * (int64_t)cv * EPV;
      T* dst = &s[cidx<T, L>(k, cv * EPV, lct, padk)];
      if (col < ncol) {
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(in + (int64_t)k * ncol + col)
                     : "memory");
      } else {
        *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else {
    for (int e = threadIdx.x; e < nk * 2 * ct; e += blockDim.x) {
      const int k = e >> (lct + 1), c2 = e & (2 * ct - 1);
      const int64_t col = c0 + c2;
      const R v = (col < ncol) ? in[(int64_t)k * ncol + col] : (R)0;
      // column 2c is the real part of working column c, column 2c + 1 the imaginary part
      R* w = reinterpret_cast<R*>(&s[cidx<T, L>(k, c2 >> 1, lct, padk)]);
      w[c2 & 1] = v;
    }
  }
  __syncthreads();
  kmesh_dft_cubic<T, L>(s, lct, padk, twc, tws);
  const R h = (R)(0.5 * scale);
  for (int e = threadIdx.x; e < nk * ct; e += blockDim.x) {
    const int k = e >> lct, c = e & (ct - 1);
    const int64_t col = c0 + 2 * (int64_t)c;
    const int j = qslot[k];
    if (col < ncol && j >= 0) {
      const int m0 = k / (L * L), m1 = (k / L) % L, m2 = k % L;
      const int km = (((L - m0) % L) * L + (L - m1) % L) * L + (L - m2) % L;
      const T zq = s[cidx<T, L>(k, c, lct, padk)], zm = s[cidx<T, L>(km, c, lct, padk)];
      T* o = out + (int64_t)j * ncol + col;
      o[0] = CT<T>::mk(h * (zq.x + zm.x), h * (zq.y - zm.y));
      if (col + 1 < ncol) o[1] = CT<T>::mk(h * (zq.y + zm.y), h * (zm.x - zq.x));
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) kdft_real_cols_kernel(const typename CT<T>::R* __restrict__ in,
                                                             T* __restrict__ out, int64_t ncol, KMesh km, int ct,
                                                             const int* __restrict__ qslot, Twiddles16 tw,
                                                             double scale) {
  using R = typename CT<T>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  __shared__ R twc[48], tws[48];
  for (int t = threadIdx.x; t < 48; t += blockDim.x) {
    twc[t] = (R)tw.c[t / 16][t % 16];
    tws[t] = (R)tw.s[t / 16][t % 16];
  }
  const int nk = km.n[0] * km.n[1] * km.n[2];
  const int64_t c0 = (int64_t)blockIdx.x * ct;
  for (int e = threadIdx.x; e < nk * ct; e += blockDim.x) {
    const int k = e / ct, c = e % ct;
    const int64_t col = c0 + c;
    const R v = (col < ncol) ? in[(int64_t)k * ncol + col] : (R)0;
    s[e] = CT<T>::mk(v, 0);
  }
  __syncthreads();
  kmesh_dft_smem<T>(s, ct, km.n, twc, tws);
  for (int e = threadIdx.x; e < nk * ct; e += blockDim.x) {
    const int k = e / ct, c = e % ct;
    const int64_t col = c0 + c;
    const int j = qslot[k];
    if (col < ncol && j >= 0) {
      const T v = s[e];
      out[(int64_t)j * ncol + col] = CT<T>::mk(v.x * (R)scale, v.y * (R)scale);
    }
  }
}

// Row padding of the cubic k-DFT's shared layout.  One 128-byte phase of a
// shared access serves G = 128 / sizeof(T) lanes; with ct < G columns per row
// those lanes span G / ct lines.  Along the stride-1 axis consecutive lines
// start L rows apart, so they land on the same banks unless the L-row group is
// padded: padk = (ct - L ct) mod G makes the line offset ct (mod G), i.e. the
// lanes of a phase cover G consecutive elements.  The other two axes step the
// line start by one row (ct elements) already.
inline int kdft_cubic_pad(int L, int ct, int elem) {
  const int G = 128 / elem;
  if (ct >= G) return 0;
  return (((ct - L * ct) % G) + G) % G;
}

template <typename T, int L, typename TS = T>
cudaError_t kdft_cubic_launch(cudaStream_t st, TS* data, int64_t ncol, int mode, const Twiddles16& t1,
                              const Twiddles16& t2, double scale) {
  constexpr int nk = L * L * L;
  int lct = 0;
  while (lct < 5 && ((int64_t)nk * sizeof(T) << (lct + 1)) <= 65536) ++lct;
  const int padk = kdft_cubic_pad(L, 1 << lct, (int)sizeof(T));
  const size_t smem = ((size_t)nk << lct) * sizeof(T) + (size_t)(nk / L) * padk * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kdft_cubic_kernel<T, L, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t nblk = (ncol + (1 << lct) - 1) >> lct;
  if (nblk > 2147483647LL) return cudaErrorInvalidValue;
  kdft_cubic_kernel<T, L, TS><<<(unsigned)nblk, 256, smem, st>>>(data, ncol, lct, padk, mode, t1, t2, scale);
  count_launch();
  return cudaGetLastError();
}

template <typename T, int L>
cudaError_t kdft_real_cubic_launch(cudaStream_t st, const typename CT<T>::R* in, T* out, int64_t ncol,
                                   const Twiddles16& tw, double scale, const int* qslot) {
  constexpr int nk = L * L * L;
  int lct = 0;
  while (lct < 5 && ((int64_t)nk * sizeof(T) << (lct + 1)) <= 65536) ++lct;
  const int padk = kdft_cubic_pad(L, 1 << lct, (int)sizeof(T));
  const size_t smem = ((size_t)nk << lct) * sizeof(T) + (size_t)(nk / L) * padk * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kdft_real_cubic_kernel<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t nblk = (ncol + (2 << lct) - 1) >> (lct + 1);  // 2 ct real columns per block
  if (nblk > 2147483647LL) return cudaErrorInvalidValue;
  // 16-byte vector loads when every row starts 16-byte aligned and a vector never
  // straddles the end of a row
  constexpr int kEpv = 16 / (int)sizeof(T);
  const int vec = ((reinterpret_cast<uintptr_t>(in) & 15) == 0 && (ncol % (2 * kEpv)) == 0 &&
                   (1 << lct) % kEpv == 0) ? 1 : 0;
  kdft_real_cubic_kernel<T, L><<<(unsigned)nblk, 256, smem, st>>>(in, out, ncol, lct, padk, qslot, tw, scale, vec);
  count_launch();
  return cudaGetLastError();
}

template <typename T, typename TS = T>
__global__ void __launch_bounds__(256) kdft_cols_kernel(TS* __restrict__ data, int64_t ncol, KMesh km,
                                                        int ct, int mode, Twiddles16 tw1,
                                                        Twiddles16 tw2, double scale) {
  using R = typename CT<T>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  __shared__ R tw1c[48], tw1s[48], tw2c[48], tw2s[48];
  for (int t = threadIdx.x; t < 48; t += blockDim.x) {
    tw1c[t] = (R)tw1.c[t / 16][t % 16];
    tw1s[t] = (R)tw1.s[t / 16][t % 16];
    tw2c[t] = (R)tw2.c[t / 16][t % 16];
    tw2s[t] = (R)tw2.s[t / 16][t % 16];
  }
  const int nk = km.n[0] * km.n[1] * km.n[2];
  const int64_t c0 = (int64_t)blockIdx.x * ct;
  for (int e = threadIdx.x; e < nk * ct; e += blockDim.x) {
    const int k = e / ct, c = e % ct;
    const int64_t col = c0 + c;
    T v = CT<T>::mk(0, 0);
    if (col < ncol) v = Cv<T, TS>::in(data[(int64_t)k * ncol + col]);
    s[e] = v;
  }
  __syncthreads();
  kmesh_dft_smem<T>(s, ct, km.n, tw1c, tw1s);
  if (mode == 1) {
    for (int e = threadIdx.x; e < nk * ct; e += blockDim.x) {
      T v = s[e];
      s[e] = CT<T>::mk(v.x * v.x + v.y * v.y, 0);
    }
    __syncthreads();
    kmesh_dft_smem<T>(s, ct, km.n, tw2c, tw2s);
  }
  for (int e = threadIdx.x; e < nk * ct; e += blockDim.x) {
    const int k = e / ct, c = e % ct;
    const int64_t col = c0 + c;
    if (col < ncol) {
      T v = s[e];
      data[(int64_t)k * ncol + col] = Cv<T, TS>::out(CT<T>::mk(v.x * (R)scale, v.y * (R)scale));
    }
  }
}

template <typename T, typename TS = T>
cudaError_t kdft_launch(cudaStream_t st, TS* data, int64_t ncol, KMesh km, int s1, int s2, int mode,
                        double scale) {
  const int nk = km.n[0] * km.n[1] * km.n[2];
  for (int a = 0; a < 3; ++a)
    if (km.n[a] < 1 || km.n[a] > 16) return cudaErrorInvalidValue;
  if (ncol <= 0) return cudaSuccess;
  if (km.n[0] == km.n[1] && km.n[1] == km.n[2]) {
    const Twiddles16 t1 = make_tw(km.n, s1), t2 = make_tw(km.n, s2);
    switch (km.n[0]) {
      case 2: return kdft_cubic_launch<T, 2, TS>(st, data, ncol, mode, t1, t2, scale);
      case 3: return kdft_cubic_launch<T, 3, TS>(st, data, ncol, mode, t1, t2, scale);
      case 4: return kdft_cubic_launch<T, 4, TS>(st, data, ncol, mode, t1, t2, scale);
      case 6: return kdft_cubic_launch<T, 6, TS>(st, data, ncol, mode, t1, t2, scale);
      case 8: return kdft_cubic_launch<T, 8, TS>(st, data, ncol, mode, t1, t2, scale);
      case 10: return kdft_cubic_launch<T, 10, TS>(st, data, ncol, mode, t1, t2, scale);
      default: break;
    }
  }
  int ct = (int)(65536 / ((int64_t)nk * sizeof(T)));
  if (ct < 1) ct = 1;
  if (ct > 32) ct = 32;
  size_t smem = (size_t)nk * ct * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kdft_cols_kernel<T, TS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int64_t nblk = (ncol + ct - 1) / ct;
  if (nblk > 2147483647LL) return cudaErrorInvalidValue;
  kdft_cols_kernel<T, TS><<<(unsigned)nblk, 256, smem, st>>>(data, ncol, km, ct, mode,
                                                         make_tw(km.n, s1), make_tw(km.n, s2), scale);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t kdft_real_launch(cudaStream_t st, const typename CT<T>::R* in, T* out, int64_t ncol, KMesh km, int s,
                             double scale, const int* qslot) {
  const int nk = km.n[0] * km.n[1] * km.n[2];
  for (int a = 0; a < 3; ++a)
    if (km.n[a] < 1 || km.n[a] > 16) return cudaErrorInvalidValue;
  if (ncol <= 0) return cudaSuccess;
  const Twiddles16 tw = make_tw(km.n, s);
  if (km.n[0] == km.n[1] && km.n[1] == km.n[2]) {
    switch (km.n[0]) {
      case 2: return kdft_real_cubic_launch<T, 2>(st, in, out, ncol, tw, scale, qslot);
      case 3: return kdft_real_cubic_launch<T, 3>(st, in, out, ncol, tw, scale, qslot);
      case 4: return kdft_real_cubic_launch<T, 4>(st, in, out, ncol, tw, scale, qslot);
      case 6: return kdft_real_cubic_launch<T, 6>(st, in, out, ncol, tw, scale, qslot);
      case 8: return kdft_real_cubic_launch<T, 8>(st, in, out, ncol, tw, scale, qslot);
      case 10: return kdft_real_cubic_launch<T, 10>(st, in, out, ncol, tw, scale, qslot);
      default: break;
    }
  }
  int ct = (int)(65536 / ((int64_t)nk * sizeof(T)));
  if (ct < 1) ct = 1;
  if (ct > 32) ct = 32;
  const size_t smem = (size_t)nk * ct * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kdft_real_cols_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t nblk = (ncol + ct - 1) / ct;
  if (nblk > 2147483647LL) return cudaErrorInvalidValue;
  kdft_real_cols_kernel<T><<<(unsigned)nblk, 256, smem, st>>>(in, out, ncol, km, ct, qslot, tw, scale);
  count_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ grid FFT
struct GridFFTParams {
  int n[3];
  int kmesh[3];
  double rec[9];
};

// Per-axis phase table: ph[a][m][g] = exp(-2 pi i m g / (nk_a n_a)), m < 16, g < 64.
__global__ void phase_table_kernel(GridFFTParams p, double2* __restrict__ ph) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 3 * 16 * 64; e += gridDim.x * blockDim.x) {
    const int a = e / 1024, m = (e / 64) % 16, g = e % 64;
    double2 v = make_double2(1.0, 0.0);
    if (m < p.kmesh[a] && g < p.n[a]) {
      const int den = p.kmesh[a] * p.n[a];
      double sn, cs;
      sincospi(-2.0 * (double)((m * g) % den) / (double)den, &sn, &cs);
      v = make_double2(cs, sn);
    }
    ph[e] = v;
  }
}

// x[row][r] *= exp(-i q.r) = ph[0][m0][g0] ph[1][m1][g1] ph[2][m2][g2]  (rows grouped by q)
template <typename T>
__global__ void phase_kernel(T* __restrict__ x, int64_t rows_per_q, int q0, int nq, GridFFTParams p,
                             const double2* __restrict__ ph) {
  using R = typename CT<T>::R;
  __shared__ T sph[3 * 16 * 64];
  for (int e = threadIdx.x; e < 3 * 16 * 64; e += blockDim.x) sph[e] = CT<T>::mk((R)ph[e].x, (R)ph[e].y);
  __syncthreads();
  const int ng = p.n[0] * p.n[1] * p.n[2];
  const int64_t total = (int64_t)nq * rows_per_q * ng;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % ng);
    const int qi = (int)(e / ((int64_t)rows_per_q * ng));
    const int q = q0 + qi;
    const int m2 = q % p.kmesh[2], m1 = (q / p.kmesh[2]) % p.kmesh[1], m0 = q / (p.kmesh[1] * p.kmesh[2]);
    const int g2 = r % p.n[2], g1 = (r / p.n[2]) % p.n[1], g0 = r / (p.n[1] * p.n[2]);
    const T f = cmul(cmul(sph[m0 * 64 + g0], sph[1024 + m1 * 64 + g1]), sph[2048 + m2 * 64 + g2]);
    x[e] = cmul(x[e], f);
  }
}

// One axis of the forward grid DFT, lines of length L with element stride S.
// Block: lpb lines x L outputs; smem holds the lines.
template <typename T>
__global__ void __launch_bounds__(256) grid_axis_kernel(T* __restrict__ x, int64_t nrows, int ng,
                                                        int L, int64_t S, int lpb,
                                                        const double2* __restrict__ tw) {
  using R = typename CT<T>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tws = reinterpret_cast<T*>(smem_raw);  // 64 twiddles in the working precision
  T* s = reinterpret_cast<T*>(smem_raw + 64 * sizeof(double2));
  const int64_t lines_per_row = ng / L;
  const int64_t total_lines = nrows * lines_per_row;
  const int64_t l0 = (int64_t)blockIdx.x * lpb;
  for (int t = threadIdx.x; t < L; t += blockDim.x) tws[t] = CT<T>::mk((R)tw[t].x, (R)tw[t].y);
  // line id -> base element offset
  auto base_of = [&](int64_t line) -> int64_t {
    const int64_t row = line / lines_per_row;
    const int64_t lr = line % lines_per_row;  // index over the other axes
    const int64_t hi = lr / S, lo = lr % S;
    return row * ng + hi * S * L + lo;
  };
  for (int e = threadIdx.x; e < lpb * L; e += blockDim.x) {
    int li, i;
    if (S == 1) {
      li = e / L;
      i = e % L;
    } else {
      li = e % lpb;
      i = e / lpb;
    }
    const int64_t line = l0 + li;
    T v = CT<T>::mk(0, 0);
    if (line < total_lines) v = x[base_of(line) + (int64_t)i * S];
    s[li * L + i] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < lpb * L; e += blockDim.x) {
    int li, j;
    if (S == 1) {
      li = e / L;
      j = e % L;
    } else {
      li = e % lpb;
      j = e / lpb;
    }
    const int64_t line = l0 + li;
    if (line >= total_lines) continue;
    const T* sl = s + li * L;
    R ax = 0, ay = 0;
    int t = 0;
    for (int i = 0; i < L; ++i) {
      const T w = tws[t];
      const T v = sl[i];
      ax += v.x * w.x - v.y * w.y;
      ay += v.x * w.y + v.y * w.x;
      t += j;
      if (t >= L) t -= L;
      if (t >= L) t %= L;
    }
    x[base_of(line) + (int64_t)j * S] = CT<T>::mk(ax, ay);
  }
}

// sw[qi][G] = sqrt(4 pi / |q+G|^2) / N_g  (0 at q+G = 0)
__global__ void weight_table_kernel(int q0, int nq, GridFFTParams p, double* __restrict__ sw) {
  const int ng = p.n[0] * p.n[1] * p.n[2];
  const int64_t total = (int64_t)nq * ng;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int h = (int)(e % ng);
    const int q = q0 + (int)(e / ng);
    const int m2 = q % p.kmesh[2], m1 = (q / p.kmesh[2]) % p.kmesh[1], m0 = q / (p.kmesh[1] * p.kmesh[2]);
    const int h2 = h % p.n[2], h1 = (h / p.n[2]) % p.n[1], h0 = h / (p.n[1] * p.n[2]);
    const int hh[3] = {h0, h1, h2};
    const int mm[3] = {m0, m1, m2};
    double fr[3];
    for (int a = 0; a < 3; ++a) {
      const int gh = (2 * hh[a] < p.n[a]) ? hh[a] : hh[a] - p.n[a];
      fr[a] = (double)mm[a] / (double)p.kmesh[a] + (double)gh;
    }
    double v2 = 0;
    for (int c = 0; c < 3; ++c) {
      const double comp = fr[0] * p.rec[0 * 3 + c] + fr[1] * p.rec[1 * 3 + c] + fr[2] * p.rec[2 * 3 + c];
      v2 += comp * comp;
    }
    const bool zero = (fr[0] == 0 && fr[1] == 0 && fr[2] == 0);
    sw[e] = zero ? 0.0 : sqrt(4.0 * M_PI / v2) / (double)ng;
  }
}

// x[qi][I][G] *= sw[qi][G]
template <typename T>
__global__ void coulomb_weight_kernel(T* __restrict__ x, int64_t rows_per_q, int nq, int ng,
                                      const double* __restrict__ sw) {
  using R = typename CT<T>::R;
  const int64_t total = (int64_t)nq * rows_per_q * ng;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int h = (int)(e % ng);
    const int64_t qi = e / ((int64_t)rows_per_q * ng);
    const R w = (R)sw[qi * ng + h];
    T v = x[e];
    x[e] = CT<T>::mk(v.x * w, v.y * w);
  }
}

template <typename T>
cudaError_t grid_fft_launch(cudaStream_t st, T* x, int rows_per_q, int q0, int nq, const CellDev& c,
                            const double2* dtw, void* work) {
  GridFFTParams p;
  for (int a = 0; a < 3; ++a) {
    p.n[a] = c.mesh[a];
    p.kmesh[a] = c.kmesh[a];
    if (c.mesh[a] < 1 || c.mesh[a] > 64) return cudaErrorInvalidValue;
  }
  for (int i = 0; i < 9; ++i) p.rec[i] = c.rec[i];
  const int ng = c.mesh[0] * c.mesh[1] * c.mesh[2];
  const int64_t nrows = (int64_t)rows_per_q * nq;
  if (nrows == 0) return cudaSuccess;
  const int64_t total = nrows * ng;
  int nb = (int)((total + 255) / 256);
  if (nb > 152 * 64) nb = 152 * 64;
  double2* ph = reinterpret_cast<double2*>(work);            // 3 x 16 x 64 phase table
  double* sw = reinterpret_cast<double*>(ph + 3 * 16 * 64);   // nq x ng weight table
  phase_table_kernel<<<12, 256, 0, st>>>(p, ph);
  count_launch();
  phase_kernel<T><<<nb, 256, 0, st>>>(x, rows_per_q, q0, nq, p, ph);
  count_launch();
  {
    int nbw = (int)(((int64_t)nq * ng + 255) / 256);
    if (nbw > 152 * 64) nbw = 152 * 64;
    weight_table_kernel<<<nbw, 256, 0, st>>>(q0, nq, p, sw);
    count_launch();
  }
  for (int a = 2; a >= 0; --a) {
    const int L = c.mesh[a];
    if (L == 1) continue;
    const int64_t S = (a == 2) ? 1 : (a == 1 ? c.mesh[2] : (int64_t)c.mesh[1] * c.mesh[2]);
    int lpb = 256 / L;
    if (lpb < 1) lpb = 1;
    const int64_t total_lines = nrows * (ng / L);
    const int64_t nblk = (total_lines + lpb - 1) / lpb;
    const size_t smem = (size_t)lpb * L * sizeof(T) + 64 * sizeof(double2);
    grid_axis_kernel<T><<<(unsigned)nblk, 256, smem, st>>>(x, nrows, ng, L, S, lpb, dtw + a * 64);
    count_launch();
  }
  coulomb_weight_kernel<T><<<nb, 256, 0, st>>>(x, rows_per_q, nq, ng, sw);
  count_launch();
  return cudaGetLastError();
}

// Z[R][(p q)][I] = conj(t[R][I][p]) t[R][I][q].  Block (p-tile of kPairP, R):
// tiles of kPairQ columns q of t[R] go through shared memory with coalesced
// loads (row pitch kPairQ + 1 against bank conflicts), and the outputs are
// written with consecutive I across threads.  Each block reads the slab t[R]
// once per p-tile from L2 and writes kPairP n_f n_p values.
constexpr int kPairP = 4, kPairQ = 16;

template <typename T>
__global__ void __launch_bounds__(256) pair_kernel(const T* __restrict__ t, int np, int nf, T* __restrict__ Z) {
  extern __shared__ __align__(16) unsigned char pair_smem[];
  T* ts = reinterpret_cast<T*>(pair_smem);  // [np][kPairQ + 1]
  const int R = blockIdx.y, p0 = blockIdx.x * kPairP;
  const T* tr = t + (int64_t)R * np * nf;
  T* zr = Z + (int64_t)R * nf * nf * np;
  for (int q0 = 0; q0 < nf; q0 += kPairQ) {
    __syncthreads();
    for (int e = threadIdx.x; e < np * kPairQ; e += blockDim.x) {
      const int I = e / kPairQ, j = e % kPairQ, q = q0 + j;
      T v;
      v.x = 0;
      v.y = 0;
      if (q < nf) v = tr[(int64_t)I * nf + q];
      ts[I * (kPairQ + 1) + j] = v;
    }
    __syncthreads();
    const int nq = min(kPairQ, nf - q0);
    for (int I = threadIdx.x; I < np; I += blockDim.x) {
#pragma unroll
      for (int pi = 0; pi < kPairP; ++pi) {
        const int p = p0 + pi;
        if (p >= nf) break;
        const T a = tr[(int64_t)I * nf + p];
        T* zp = zr + ((int64_t)p * nf + q0) * np + I;
        for (int j = 0; j < nq; ++j) {
          const T b = ts[I * (kPairQ + 1) + j];
          T z;
          z.x = a.x * b.x + a.y * b.y;  // conj(a) b
          z.y = a.x * b.y - a.y * b.x;
          zp[(int64_t)j * np] = z;
        }
      }
    }
  }
}

// Pair rows in the time-reversal basis, real:  for the pair o = (p, q), p < q
// (lexicographic), row 2o = 2 Re(conj(t_p) t_q) and row 2o + 1 = 2 Im(conj(t_p) t_q)
// (the combinations Z_(pq) + Z_(qp) and -i (Z_(pq) - Z_(qp))), and row 2P + p = |t_p|^2.
// Zr[R][row][I]; same block structure as pair_kernel (one R and kPairP values of p per
// block, 16-column tiles of t[R] through shared memory, I across threads).
template <typename T>
__global__ void __launch_bounds__(256) pair_real_kernel(const T* __restrict__ t, int np, int nf,
                                                        typename CT<T>::R* __restrict__ Zr, int64_t row0,
                                                        int64_t rows) {
  using R = typename CT<T>::R;
  extern __shared__ __align__(16) unsigned char pair_smem[];
  T* ts = reinterpret_cast<T*>(pair_smem);  // [np][kPairQ + 1]
  const int Rk = blockIdx.y, p0 = blockIdx.x * kPairP;
  const int64_t P = (int64_t)nf * (nf - 1) / 2;
  const T* tr = t + (int64_t)Rk * np * nf;
  R* zr = Zr + ((int64_t)Rk * rows + row0) * np;
  for (int q0 = p0; q0 < nf; q0 += kPairQ) {
    __syncthreads();
    for (int e = threadIdx.x; e < np * kPairQ; e += blockDim.x) {
      const int I = e / kPairQ, j = e % kPairQ, q = q0 + j;
      T v;
      v.x = 0;
      v.y = 0;
      if (q < nf) v = tr[(int64_t)I * nf + q];
      ts[I * (kPairQ + 1) + j] = v;
    }
    __syncthreads();
    const int nq = min(kPairQ, nf - q0);
    for (int I = threadIdx.x; I < np; I += blockDim.x) {
#pragma unroll
      for (int pi = 0; pi < kPairP; ++pi) {
        const int p = p0 + pi;
        if (p >= nf) break;
        const T a = tr[(int64_t)I * nf + p];
        const int64_t o0 = (int64_t)p * nf - (int64_t)p * (p + 1) / 2 - p - 1;  // pair index of (p, q) is o0 + q
        for (int j = 0; j < nq; ++j) {
          const int q = q0 + j;
          if (q < p) continue;
          const T b = ts[I * (kPairQ + 1) + j];
          if (q == p) {
            zr[(2 * P + p) * np + I] = a.x * a.x + a.y * a.y;
          } else {
            const int64_t o = o0 + q;
            zr[(2 * o) * np + I] = (R)2 * (a.x * b.x + a.y * b.y);      // 2 Re(conj(a) b)
            zr[(2 * o + 1) * np + I] = (R)2 * (a.x * b.y - a.y * b.x);  // 2 Im(conj(a) b)
          }
        }
      }
    }
  }
}

template <typename T>
cudaError_t pair_launch(cudaStream_t st, const T* t, int nk, int np, int nf, T* Z) {
  if ((int64_t)nk * nf * np == 0) return cudaSuccess;
  if (nk > 65535) return cudaErrorInvalidValue;
  const size_t smem = (size_t)np * (kPairQ + 1) * sizeof(T);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(pair_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  pair_kernel<T><<<dim3((nf + kPairP - 1) / kPairP, nk), 256, smem, st>>>(t, np, nf, Z);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t pair_real_launch(cudaStream_t st, const T* t, int nk, int np, int nf, typename CT<T>::R* Zr,
                             int64_t row0, int64_t rows) {
  if ((int64_t)nk * nf * np == 0) return cudaSuccess;
  if (nk > 65535) return cudaErrorInvalidValue;
  const size_t smem = (size_t)np * (kPairQ + 1) * sizeof(T);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(pair_real_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  pair_real_kernel<T><<<dim3((nf + kPairP - 1) / kPairP, nk), 256, smem, st>>>(t, np, nf, Zr, row0, rows);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t kdft_real_f(cudaStream_t st, const float* in, float2* out, int64_t ncol, KMesh km, int s, float scale,
                        const int* qslot) {
  return kdft_real_launch<float2>(st, in, out, ncol, km, s, scale, qslot);
}
cudaError_t pair_products_real_f(cudaStream_t st, const float2* t, int nk, int np, int nf, float* Zr, int64_t row0,
                                 int64_t rows) {
  if (row0 < 0 || row0 + (int64_t)nf * nf > rows) return cudaErrorInvalidValue;
  return pair_real_launch<float2>(st, t, nk, np, nf, Zr, row0, rows);
}

cudaError_t kdft_cols(cudaStream_t st, double2* data, int64_t ncol, KMesh km, int s1, int s2,
                      int mode, double scale) {
  return kdft_launch<double2>(st, data, ncol, km, s1, s2, mode, scale);
}
cudaError_t kdft_cols_f(cudaStream_t st, float2* data, int64_t ncol, KMesh km, int s1, int s2,
                        int mode, float scale) {
  return kdft_launch<float2>(st, data, ncol, km, s1, s2, mode, scale);
}
size_t grid_coulomb_work_bytes(int nq, const CellDev& c) {
  return 3 * 16 * 64 * sizeof(double2) + (size_t)nq * c.mesh[0] * c.mesh[1] * c.mesh[2] * sizeof(double);
}
cudaError_t grid_coulomb_fft(cudaStream_t st, double2* x, int rows_per_q, int q0, int nq,
                             const CellDev& c, const double2* dtw, void* work) {
  return grid_fft_launch<double2>(st, x, rows_per_q, q0, nq, c, dtw, work);
}
cudaError_t grid_coulomb_fft_f(cudaStream_t st, float2* x, int rows_per_q, int q0, int nq,
                               const CellDev& c, const double2* dtw, void* work) {
  return grid_fft_launch<float2>(st, x, rows_per_q, q0, nq, c, dtw, work);
}
cudaError_t grid_coulomb_fft_ff(cudaStream_t st, ffcomplex* x, int rows_per_q, int q0, int nq,
                                const CellDev& c, const double2* dtw, void* work) {
  return grid_fft_launch<ffcomplex>(st, x, rows_per_q, q0, nq, c, dtw, work);
}

void grid_twiddles(const int mesh[3], double2* host192) {
  for (int a = 0; a < 3; ++a)
    for (int j = 0; j < 64; ++j) {
      double ang = j < mesh[a] ? 2.0 * M_PI * j / mesh[a] : 0.0;
      host192[a * 64 + j] = make_double2(std::cos(ang), -std::sin(ang));
    }
}
cudaError_t pair_products(cudaStream_t st, const double2* t, int nk, int np, int nf, double2* Z) {
  return pair_launch<double2>(st, t, nk, np, nf, Z);
}

// ---- float-float variants (FP64-class tensor-core path)
namespace {
__global__ void z2ff_kernel(const double2* __restrict__ in, ffcomplex* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = in[e];
    out[e] = ffcomplex{ffloat(v.x), ffloat(v.y)};
  }
}
}  // namespace

cudaError_t z2ff(cudaStream_t st, const double2* in, ffcomplex* out, int64_t n) {
  if (n <= 0) return cudaSuccess;
  int64_t nb = (n + 255) / 256;
  if (nb > 152 * 32) nb = 152 * 32;
  z2ff_kernel<<<(unsigned)nb, 256, 0, st>>>(in, out, n);
  count_launch();
  return cudaGetLastError();
}
cudaError_t kdft_cols_ff(cudaStream_t st, ffcomplex* data, int64_t ncol, KMesh km, int s1, int s2, int mode,
                         double scale) {
  return kdft_launch<ffcomplex>(st, data, ncol, km, s1, s2, mode, scale);
}
cudaError_t kdft_cols_zff(cudaStream_t st, double2* data, int64_t ncol, KMesh km, int s1, int s2, int mode,
                          double scale) {
  return kdft_launch<ffcomplex, double2>(st, data, ncol, km, s1, s2, mode, scale);
}
cudaError_t kdft_real_ff(cudaStream_t st, const ffloat* in, ffcomplex* out, int64_t ncol, KMesh km, int s,
                         double scale, const int* qslot) {
  return kdft_real_launch<ffcomplex>(st, in, out, ncol, km, s, scale, qslot);
}
cudaError_t pair_products_real_ff(cudaStream_t st, const ffcomplex* t, int nk, int np, int nf, ffloat* Zr,
                                  int64_t row0, int64_t rows) {
  if (row0 < 0 || row0 + (int64_t)nf * nf > rows) return cudaErrorInvalidValue;
  return pair_real_launch<ffcomplex>(st, t, nk, np, nf, Zr, row0, rows);
}

}  // namespace isdf
