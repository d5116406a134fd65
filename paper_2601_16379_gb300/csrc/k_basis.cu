// Crystalline Gaussian orbitals on the cell grid (Eq. 1) and the
// interpolation-point selection of Section II.A.
//
// ao_eval   Phi^k_mu(r) = sum_T e^{i k.T} phi~_mu(r - T), T over the box
//           |n_i| <= L_i.  For orthorhombic cells the Gaussian and the phase
//           factorise per axis, so the box sum is the product of three 1-D
//           lattice sums S_a(m_a, g_a) per primitive (exactly the same terms as
//           the 3-D box).  Other cells use a direct 3-D sum.
// ip_*      greedy pivoted Cholesky of K(r,r') = D(r,r')^2 with
//           D(r,r') = Re sum_{k,mu} conj(Phi^k_mu(r)) Phi^k_mu(r') (D is real:
//           the k and -k terms are conjugate).  One pivot per ip_step: argmax
//           with ties, column generation, rank-one update.
#include <cmath>

#include "common.cuh"

namespace isdf {

namespace {

constexpr int KCH = 8;  // k-points per thread in the general path

// --------------------------------------------------------- orthorhombic path
// S[((mu*maxprim + p)*3 + a)*16*64 + m*64 + g] = sum_n e^{2 pi i m n/nk_a} x^l e^{-alpha x^2},
// x = g a_a/n_a - A_a - n a_a.
__global__ void ao_1d_kernel(CellDev c, BasisDev b, double2* __restrict__ S) {
  const int total = b.nao * b.maxprim * 3 * 16 * 64;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int g = e % 64;
    const int m = (e / 64) % 16;
    const int a = (e / (64 * 16)) % 3;
    const int p = (e / (64 * 16 * 3)) % b.maxprim;
    const int mu = e / (64 * 16 * 3 * b.maxprim);
    double2 acc = make_double2(0.0, 0.0);
    const int sh = b.ao_shell[mu];
    const int np = b.sh_off[sh + 1] - b.sh_off[sh];
    if (g < c.mesh[a] && m < c.kmesh[a] && p < np) {
      const double alpha = b.prim_exp[b.sh_off[sh] + p];
      const int l = b.ao_lxyz[mu * 3 + a];
      const double La = c.lat[a * 3 + a];
      const double A = b.coords[b.sh_atom[sh] * 3 + a];
      const double r = (double)g * La / (double)c.mesh[a];
      for (int n = -c.lrange[a]; n <= c.lrange[a]; ++n) {
        const double x = r - A - (double)n * La;
        double v = exp(-alpha * x * x);
        for (int t = 0; t < l; ++t) v *= x;
        // phase e^{2 pi i m n / nk}, angle reduced exactly
        const int nk = c.kmesh[a];
        int mn = (m * n) % nk;
        if (mn < 0) mn += nk;
        double sn, cs;
        sincospi(2.0 * (double)mn / (double)nk, &sn, &cs);
        acc.x += cs * v;
        acc.y += sn * v;
      }
    }
    S[e] = acc;
  }
}

__global__ void ao_combine_kernel(CellDev c, BasisDev b, const double2* __restrict__ S,
                                  double2* __restrict__ phi) {
  const int ng = c.mesh[0] * c.mesh[1] * c.mesh[2];
  const int nk = c.kmesh[0] * c.kmesh[1] * c.kmesh[2];
  const int64_t total = (int64_t)nk * b.nao * ng;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % ng);
    const int mu = (int)((e / ng) % b.nao);
    const int k = (int)(e / ((int64_t)ng * b.nao));
    const int g2 = r % c.mesh[2], g1 = (r / c.mesh[2]) % c.mesh[1], g0 = r / (c.mesh[1] * c.mesh[2]);
    const int m2 = k % c.kmesh[2], m1 = (k / c.kmesh[2]) % c.kmesh[1], m0 = k / (c.kmesh[1] * c.kmesh[2]);
    const int sh = b.ao_shell[mu];
    const int np = b.sh_off[sh + 1] - b.sh_off[sh];
    double2 acc = make_double2(0.0, 0.0);
    for (int p = 0; p < np; ++p) {
      const double2* base = S + (int64_t)((mu * b.maxprim + p) * 3) * 16 * 64;
      const double2 sx = base[0 * 1024 + m0 * 64 + g0];
      const double2 sy = base[1 * 1024 + m1 * 64 + g1];
      const double2 sz = base[2 * 1024 + m2 * 64 + g2];
      const double cn = b.prim_norm[mu * b.maxprim + p];
      const double2 t = cmul(cmul(sx, sy), sz);
      acc.x += cn * t.x;
      acc.y += cn * t.y;
    }
    phi[e] = acc;
  }
}

// ------------------------------------------------------------- general path
__global__ void ao_general_kernel(CellDev c, BasisDev b, double2* __restrict__ phi) {
  const int ng = c.mesh[0] * c.mesh[1] * c.mesh[2];
  const int nk = c.kmesh[0] * c.kmesh[1] * c.kmesh[2];
  const int nkc = (nk + KCH - 1) / KCH;
  const int64_t total = (int64_t)nkc * b.nao * ng;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % ng);
    const int mu = (int)((e / ng) % b.nao);
    const int kc = (int)(e / ((int64_t)ng * b.nao));
    const int g2 = r % c.mesh[2], g1 = (r / c.mesh[2]) % c.mesh[1], g0 = r / (c.mesh[1] * c.mesh[2]);
    const double f[3] = {(double)g0 / c.mesh[0], (double)g1 / c.mesh[1], (double)g2 / c.mesh[2]};
    double rc[3];
    for (int x = 0; x < 3; ++x) rc[x] = f[0] * c.lat[0 * 3 + x] + f[1] * c.lat[1 * 3 + x] + f[2] * c.lat[2 * 3 + x];
    const int sh = b.ao_shell[mu];
    const int np = b.sh_off[sh + 1] - b.sh_off[sh];
    const int lx = b.ao_lxyz[mu * 3], ly = b.ao_lxyz[mu * 3 + 1], lz = b.ao_lxyz[mu * 3 + 2];
    const double* A = b.coords + b.sh_atom[sh] * 3;
    double2 acc[KCH];
    int km[KCH][3];
    for (int i = 0; i < KCH; ++i) {
      acc[i] = make_double2(0.0, 0.0);
      const int k = kc * KCH + i;
      const int kk = k < nk ? k : 0;
      km[i][2] = kk % c.kmesh[2];
      km[i][1] = (kk / c.kmesh[2]) % c.kmesh[1];
      km[i][0] = kk / (c.kmesh[1] * c.kmesh[2]);
    }
    for (int n0 = -c.lrange[0]; n0 <= c.lrange[0]; ++n0)
      for (int n1 = -c.lrange[1]; n1 <= c.lrange[1]; ++n1)
        for (int n2 = -c.lrange[2]; n2 <= c.lrange[2]; ++n2) {
          double d[3];
          for (int x = 0; x < 3; ++x)
            d[x] = rc[x] - A[x] - (n0 * c.lat[0 * 3 + x] + n1 * c.lat[1 * 3 + x] + n2 * c.lat[2 * 3 + x]);
          const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          double poly = 1.0;
          for (int t = 0; t < lx; ++t) poly *= d[0];
          for (int t = 0; t < ly; ++t) poly *= d[1];
          for (int t = 0; t < lz; ++t) poly *= d[2];
          double v = 0.0;
          for (int p = 0; p < np; ++p)
            v += b.prim_norm[mu * b.maxprim + p] * exp(-b.prim_exp[b.sh_off[sh] + p] * r2);
          v *= poly;
          for (int i = 0; i < KCH; ++i) {
            // e^{2 pi i sum_a m_a n_a / nk_a}
            double fr = 0.0;
            const int nn[3] = {n0, n1, n2};
            for (int a = 0; a < 3; ++a) {
              int mn = (km[i][a] * nn[a]) % c.kmesh[a];
              if (mn < 0) mn += c.kmesh[a];
              fr += (double)mn / (double)c.kmesh[a];
            }
            double sn, cs;
            sincospi(2.0 * (fr - floor(fr)), &sn, &cs);
            acc[i].x += cs * v;
            acc[i].y += sn * v;
          }
        }
    for (int i = 0; i < KCH; ++i) {
      const int k = kc * KCH + i;
      if (k < nk) phi[((int64_t)k * b.nao + mu) * ng + r] = acc[i];
    }
  }
}

// ------------------------------------------------------------- IP selection
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// partial[s][r] = sum_{a in split s} Re(conj(F[a][r]) F[a][col]) ; col < 0 -> |F[a][r]|^2
__global__ void ip_partial_kernel(const double2* __restrict__ F, int nkao, int ng,
                                  const int32_t* __restrict__ pcol_ptr, int j, int nsplit,
                                  double* __restrict__ partial, const int32_t* __restrict__ status) {
  if (status && *status != 0) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (r >= ng) return;
  const int per = (nkao + nsplit - 1) / nsplit;
  const int a0 = s * per, a1 = min(nkao, a0 + per);
  const int p = pcol_ptr ? pcol_ptr[j] : -1;
  double acc0 = 0.0, acc1 = 0.0;
  int a = a0;
  if (p >= 0) {
    for (; a + 1 < a1; a += 2) {
      const double2 x0 = F[(int64_t)a * ng + r], y0 = F[(int64_t)a * ng + p];
      const double2 x1 = F[(int64_t)(a + 1) * ng + r], y1 = F[(int64_t)(a + 1) * ng + p];
      acc0 = fma(x0.x, y0.x, acc0);
      acc0 = fma(x0.y, y0.y, acc0);
      acc1 = fma(x1.x, y1.x, acc1);
      acc1 = fma(x1.y, y1.y, acc1);
    }
    for (; a < a1; ++a) {
      const double2 x0 = F[(int64_t)a * ng + r], y0 = F[(int64_t)a * ng + p];
      acc0 = fma(x0.x, y0.x, acc0);
      acc0 = fma(x0.y, y0.y, acc0);
    }
  } else {
    for (; a < a1; ++a) {
      const double2 x0 = F[(int64_t)a * ng + r];
      acc0 = fma(x0.x, x0.x, acc0);
      acc0 = fma(x0.y, x0.y, acc0);
    }
  }
  partial[(int64_t)s * ng + r] = acc0 + acc1;
}

__global__ void ip_init_combine_kernel(const double* __restrict__ partial, int nsplit, int ng,
                                       double* __restrict__ d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ng) return;
  double D = 0.0;
  for (int s = 0; s < nsplit; ++s) D += partial[(int64_t)s * ng + r];
  d[r] = D * D;
}

// Single block: argmax with the tie rule; writes piv[j], chosen, dp (= d[p]).
__global__ void __launch_bounds__(1024) ip_argmax_kernel(const double* __restrict__ d, int ng, int j,
                                                         int32_t* __restrict__ piv,
                                                         int32_t* __restrict__ chosen,
                                                         uint64_t seed, double tie_eps,
                                                         double chol_tol, double* __restrict__ scal,
                                                         int32_t* __restrict__ status) {
  // scal[0] = d0 (set on j == 0), scal[1] = d[p] of the current pivot
  __shared__ double sv[32];
  __shared__ unsigned long long sh[32];
  __shared__ int si[32];
  __shared__ double s_dmax;
  if (*status != 0) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  double m = -INFINITY;
  for (int r = tid; r < ng; r += blockDim.x)
    if (!chosen[r]) m = fmax(m, d[r]);
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) sv[w] = m;
  __syncthreads();
  if (w == 0) {
    double v = lane < (int)(blockDim.x >> 5) ? sv[lane] : -INFINITY;
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) s_dmax = v;
  }
  __syncthreads();
  const double dmax = s_dmax;
  if (j == 0 && tid == 0) scal[0] = dmax;
  const double d0 = (j == 0) ? dmax : scal[0];
  if (!(dmax >= chol_tol * d0) || !(dmax > 0.0)) {
    if (tid == 0) {
      *status = 1;
      piv[j] = -1;
    }
    return;
  }
  const double thr = fmax(dmax - tie_eps * d0, 0.5 * dmax);
  unsigned long long best = ~0ULL;
  int bi = -1;
  for (int r = tid; r < ng; r += blockDim.x) {
    if (chosen[r] || !(d[r] >= thr)) continue;
    const unsigned long long hsh = splitmix64(seed ^ (uint64_t)r);
    if (hsh < best || (hsh == best && r < bi)) {
      best = hsh;
      bi = r;
    }
  }
  for (int o = 16; o; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob < best || (ob == best && oi >= 0 && (bi < 0 || oi < bi))) {
      best = ob;
      bi = oi;
    }
  }
  if (lane == 0) {
    sh[w] = best;
    si[w] = bi;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long b = ~0ULL;
    int p = -1;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i)
      if (si[i] >= 0 && (sh[i] < b || (sh[i] == b && si[i] < p))) {
        b = sh[i];
        p = si[i];
      }
    if (p < 0) {
      *status = 2;
      piv[j] = -1;
      return;
    }
    piv[j] = p;
    chosen[p] = 1;
    scal[1] = d[p];
  }
}

// l_r = (D(r,p)^2 - sum_{i<j} Lt[i][r] Lt[i][p]) / sqrt(d_p);  d_r -= l_r^2
__global__ void ip_update_kernel(const double* __restrict__ partial, int nsplit, int ng, int j,
                                 const int32_t* __restrict__ piv, double* __restrict__ Lt,
                                 double* __restrict__ d, const double* __restrict__ scal,
                                 const int32_t* __restrict__ status) {
  if (*status != 0) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ng) return;
  const int p = piv[j];
  double D = 0.0;
  for (int s = 0; s < nsplit; ++s) D += partial[(int64_t)s * ng + r];
  double acc = D * D;
  for (int i = 0; i < j; ++i) acc -= Lt[(int64_t)i * ng + r] * Lt[(int64_t)i * ng + p];
  const double l = acc / sqrt(scal[1]);
  Lt[(int64_t)j * ng + r] = l;
  d[r] -= l * l;
}

__global__ void gather_x_kernel(const double2* __restrict__ phi, int nk, int nao, int ng,
                                const int32_t* __restrict__ ips, int np, double2* __restrict__ X) {
  const int64_t total = (int64_t)nk * np * nao;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int mu = (int)(e % nao);
    const int I = (int)((e / nao) % np);
    const int k = (int)(e / ((int64_t)nao * np));
    X[e] = phi[((int64_t)k * nao + mu) * ng + ips[I]];
  }
}

inline int nblocks(int64_t total, int cap = 152 * 32) {
  int64_t nb = (total + 255) / 256;
  if (nb > cap) nb = cap;
  if (nb < 1) nb = 1;
  return (int)nb;
}

}  // namespace

size_t ao_eval_work_bytes(const CellDev&, const BasisDev& b) {
  return (size_t)b.nao * b.maxprim * 3 * 16 * 64 * sizeof(double2);
}

cudaError_t ao_eval(cudaStream_t st, const CellDev& c, const BasisDev& b, double2* phi, double* work) {
  const int ng = c.mesh[0] * c.mesh[1] * c.mesh[2];
  const int nk = c.kmesh[0] * c.kmesh[1] * c.kmesh[2];
  if (c.orthorhombic) {
    double2* S = reinterpret_cast<double2*>(work);
    const int total1 = b.nao * b.maxprim * 3 * 16 * 64;
    ao_1d_kernel<<<nblocks(total1), 256, 0, st>>>(c, b, S);
    count_launch();
    ao_combine_kernel<<<nblocks((int64_t)nk * b.nao * ng), 256, 0, st>>>(c, b, S, phi);
    count_launch();
  } else {
    const int64_t total = (int64_t)((nk + KCH - 1) / KCH) * b.nao * ng;
    ao_general_kernel<<<nblocks(total, 152 * 16), 256, 0, st>>>(c, b, phi);
    count_launch();
  }
  return cudaGetLastError();
}

cudaError_t ip_init(cudaStream_t st, const double2* phi, int nkao, int ng, double* d, double* partial) {
  const int nsplit = 16;
  dim3 g((ng + 255) / 256, nsplit);
  ip_partial_kernel<<<g, 256, 0, st>>>(phi, nkao, ng, nullptr, 0, nsplit, partial, nullptr);
  count_launch();
  ip_init_combine_kernel<<<(ng + 255) / 256, 256, 0, st>>>(partial, nsplit, ng, d);
  count_launch();
  return cudaGetLastError();
}

cudaError_t ip_step(cudaStream_t st, const double2* phi, int nkao, int ng, int j, double* d, double* Lt,
                    int32_t* piv, int32_t* chosen, double* partial, int nsplit, uint64_t seed,
                    double tie_eps, double chol_tol, double* scal, int32_t* status) {
  ip_argmax_kernel<<<1, 1024, 0, st>>>(d, ng, j, piv, chosen, seed, tie_eps, chol_tol, scal, status);
  count_launch();
  dim3 g((ng + 255) / 256, nsplit);
  ip_partial_kernel<<<g, 256, 0, st>>>(phi, nkao, ng, piv, j, nsplit, partial, status);
  count_launch();
  ip_update_kernel<<<(ng + 255) / 256, 256, 0, st>>>(partial, nsplit, ng, j, piv, Lt, d, scal, status);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gather_x(cudaStream_t st, const double2* phi, int nk, int nao, int ng, const int32_t* ips,
                     int np, double2* X) {
  gather_x_kernel<<<nblocks((int64_t)nk * np * nao), 256, 0, st>>>(phi, nk, nao, ng, ips, np, X);
  count_launch();
  return cudaGetLastError();
}

}  // namespace isdf
