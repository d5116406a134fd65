// Internal declarations shared by the CUDA translation units of libisdf.
// Complex128 is double2 (x = re, y = im); complex64 is float2.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "ff.cuh"

namespace isdf {

// ---------------------------------------------------------------- complex ops
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) {
  return make_double2(a.x * s, a.y * s);
}
// acc += a * b
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// ------------------------------------------------------------- launch errors
struct Err {
  int code = 0;
  std::string msg;
};

// Counts kernel launches made through the library (for launch accounting).
extern thread_local int64_t* g_launch_counter;
inline void count_launch() {
  if (g_launch_counter) ++*g_launch_counter;
}

// ------------------------------------------------------------------- kernels
// Batched complex GEMM, row-major: C_b = alpha * op(A_b) op(B_b) + beta * C_b.
// op: 'N' as is, 'T' transpose, 'C' conjugate transpose, 'R' conjugate only.
cudaError_t zgemm(cudaStream_t st, char opA, char opB, int m, int n, int k, double2 alpha,
                  const double2* A, int64_t lda, int64_t sA, const double2* B, int64_t ldb,
                  int64_t sB, double2 beta, double2* C, int64_t ldc, int64_t sC, int batch);
// C_b = A_b * gather_rows(B_b, brow_b) with A_b (m x m) lower triangular: the
// k > row blocks are skipped.  Rows with brow < 0 contribute zero.
cudaError_t ztrmm_gather(cudaStream_t st, int m, int n, const double2* A, int64_t lda, int64_t sA,
                         const int32_t* brow, int64_t sIdx, const double2* B, int64_t ldb, int64_t sB, double2* C,
                         int64_t ldc, int64_t sC, int batch);
cudaError_t cgemm(cudaStream_t st, char opA, char opB, int m, int n, int k, float2 alpha,
                  const float2* A, int64_t lda, int64_t sA, const float2* B, int64_t ldb,
                  int64_t sB, float2 beta, float2* C, int64_t ldc, int64_t sC, int batch);

// k-mesh DFT along the leading (k) axis of data[Nk][ncol] (complex128), in place.
//   mode 0: data = scale * DFT_s1(data)
//   mode 1: data = scale * DFT_s2(|DFT_s1(data)|^2)
// s = +1 means sum_k exp(+2 pi i m.k/nk), s = -1 the opposite sign.
struct KMesh {
  int n[3];
};
cudaError_t kdft_cols(cudaStream_t st, double2* data, int64_t ncol, KMesh km, int s1, int s2,
                      int mode, double scale);
cudaError_t kdft_cols_f(cudaStream_t st, float2* data, int64_t ncol, KMesh km, int s1, int s2,
                        int mode, float scale);

// Bloch AO values phi[k][mu][r] (complex128).
struct BasisDev {
  int nao;
  int nshell;
  const int* ao_shell;      // [nao] shell of each AO
  const int* ao_lxyz;       // [nao*3]
  const int* sh_atom;       // [nshell]
  const int* sh_off;        // [nshell+1] primitive offsets
  const double* prim_exp;   // [nprim]
  const double* prim_cn;    // [nprim*ncomp?] coef * norm for component 0 (radial)
  const double* prim_norm;  // [nao * maxprim] coef*norm per AO and primitive
  const double* coords;     // [natm*3]
  int maxprim;
};
struct CellDev {
  double lat[9];
  double rec[9];
  int kmesh[3];
  int mesh[3];
  int lrange[3];
  double expcut;
  int orthorhombic;
};
cudaError_t ao_eval(cudaStream_t st, const CellDev& c, const BasisDev& b, double2* phi,
                    double* work1d);
size_t ao_eval_work_bytes(const CellDev& c, const BasisDev& b);

// IP selection.
cudaError_t ip_init(cudaStream_t st, const double2* phi, int nkao, int ng, double* d,
                    double* dscratch);
cudaError_t ip_step(cudaStream_t st, const double2* phi, int nkao, int ng, int j, double* d,
                    double* Lt, int32_t* piv, int32_t* chosen, double* partial, int nsplit,
                    uint64_t seed, double tie_eps, double chol_tol, double* d0, int32_t* status);
cudaError_t gather_x(cudaStream_t st, const double2* phi, int nk, int nao, int ng,
                     const int32_t* ips, int np, double2* X);

// Pivoted Cholesky (batched) of Hermitian PSD A[b][n][n].  Lt[b][j][i] = L[i][j].
cudaError_t pchol_batched(cudaStream_t st, const double2* A, int n, int batch, double tol,
                          double2* Lt, int32_t* perm, int32_t* rank, double* dwork);
// Wfull[b] (n x n): Wfull[i][perm[c]] = (L_S^{-1})[i][c], zero elsewhere.
cudaError_t trinv_batched(cudaStream_t st, const double2* Lt, const int32_t* perm,
                          const int32_t* rank, int n, int batch, double2* W, double2* work);
// Lpad[b][i][j] = L[i][j] (row-major, columns beyond the rank zero).
cudaError_t lt_to_rowmajor(cudaStream_t st, const double2* Lt, const int32_t* rank, int n,
                           int batch, double2* L);

// Grid FFT of rows x[q][I][r] (complex128), in place:
//   x <- sqrt(w(q+G)) * (1/N_g) FFT(e^{-i q.r} x)   with w = 4 pi/|q+G|^2, 0 at q+G = 0.
// dtw: device table of 3 x 64 forward twiddles exp(-2 pi i j/n_a) (grid_twiddles);
// work: grid_coulomb_work_bytes(nq) bytes of device scratch (phase and weight tables).
size_t grid_coulomb_work_bytes(int nq, const CellDev& c);
cudaError_t grid_coulomb_fft(cudaStream_t st, double2* x, int rows_per_q, int q0, int nq,
                             const CellDev& c, const double2* dtw, void* work);
cudaError_t grid_coulomb_fft_f(cudaStream_t st, float2* x, int rows_per_q, int q0, int nq,
                               const CellDev& c, const double2* dtw, void* work);
// the same in float-float (FP32 arithmetic, ~2^-44), in place on float-float data
cudaError_t grid_coulomb_fft_ff(cudaStream_t st, ffcomplex* x, int rows_per_q, int q0, int nq,
                                const CellDev& c, const double2* dtw, void* work);
void grid_twiddles(const int mesh[3], double2* host192);

// Real k-mesh DFT out of place, keeping the q with qslot[q] >= 0 (complex64 output):
//   out[qslot[q]][col] = scale sum_k e^{s 2 pi i m_q.m_k/n} in[k][col].
cudaError_t kdft_real_f(cudaStream_t st, const float* in, float2* out, int64_t ncol, KMesh km, int s, float scale,
                        const int* qslot);
// Real pair rows of the time-reversal basis: for pairs o = (p < q) in lexicographic
// order Zr[R][2o][I] = 2 Re(conj(t_p) t_q), Zr[R][2o+1][I] = 2 Im(conj(t_p) t_q), and
// Zr[R][2P + p][I] = |t_p|^2 (P = n_f (n_f - 1)/2), t = t[R][I][p] complex64.
// Rows row0 .. row0 + n_f^2 - 1 of a stack of `rows` rows: Zr[R][row0 + row][I].
cudaError_t pair_products_real_f(cudaStream_t st, const float2* t, int nk, int np, int nf, float* Zr, int64_t row0,
                                 int64_t rows);
// Float-float variants for the FP64-class tensor-core path (ff.cuh): the k -> R
// DFT of T, the real pair rows and their R -> q DFT, in FP32 arithmetic at ~2^-44.
cudaError_t z2ff(cudaStream_t st, const double2* in, ffcomplex* out, int64_t n);
cudaError_t kdft_cols_ff(cudaStream_t st, ffcomplex* data, int64_t ncol, KMesh km, int s1, int s2, int mode,
                         double scale);
// complex128 data transformed in float-float (as kdft_cols, ~2^-44 relative)
cudaError_t kdft_cols_zff(cudaStream_t st, double2* data, int64_t ncol, KMesh km, int s1, int s2, int mode,
                          double scale);
cudaError_t kdft_real_ff(cudaStream_t st, const ffloat* in, ffcomplex* out, int64_t ncol, KMesh km, int s,
                         double scale, const int* qslot);
cudaError_t pair_products_real_ff(cudaStream_t st, const ffcomplex* t, int nk, int np, int nf, ffloat* Zr,
                                  int64_t row0, int64_t rows);
// Fragment pair products Z[R][(p q)][I] = conj(t[R][I][p]) * t[R][I][q].
cudaError_t pair_products(cudaStream_t st, const double2* t, int nk, int np, int nf, double2* Z);

// eri[p][q][r][s] = E[(p q)][(s r)] * scale, and the traces.
cudaError_t eri_permute(cudaStream_t st, const double2* E, int nf, double scale, double2* eri);
cudaError_t eri_traces(cudaStream_t st, const double2* E, int nf, double scale,
                       const double2* gamma, double* out4, double2* part);

// Message of the last failed handle-free call on this thread.
const char* noalloc_last_error();

// Tensor-core E = sum_q B^q B^q^H (k_tc.cu) in the real symmetric form of the
// time-reversal basis.  The rows of B are those of that basis (pair o = (p < q) ->
// rows 2o, 2o + 1; diagonal p -> row 2P + p), addressed as
// (a, k = Q nJ + J) -> B[slot(Q) sQ + a sA + J] with slot(Q) = qmap[Q] (or Q when
// qmap is NULL), J < nJ, over the nS positions of the sum.  Row exponents over
// all positions, then each chunk of positions (accumulate = 0 for the first),
// then the finish (E = W E' W^H times scale, written as the chemist-order ERIs
// with the traces on the way); orb: the orbits of pair_orbits (device copy,
// n_f (n_f+1)/2 entries).
void pair_orbits(int nf, std::vector<int2>& orb);
size_t syrk_tc_split_bytes(int64_t n2, int64_t kcols);
void syrk_tc_tiles(int64_t n2, std::vector<int2>& tiles, std::vector<int>& tile_of, int band = 12);
size_t syrk_tc_ws_bytes(int64_t ntiles);
cudaError_t syrk_tc_rowscale(cudaStream_t st, const float2* B, int64_t sQ, int64_t sA, int64_t nJ, const int* qmap,
                             int nS, int64_t n2, int* row_exp);
// cfg selects the pipeline of the tile kernel: 0 = K rows of 64 fp16 (128-byte
// swizzle), 3 stages; 1 = rows of 32 fp16 (64-byte swizzle), 6 stages.
cudaError_t syrk_tc_chunk(cudaStream_t st, const float2* B, int64_t sQ, int64_t sA, int64_t nJ, const int* qmap,
                          int64_t n2, int j0, int nq, const int* row_exp, void* split, const int2* tiles_d, int ntiles,
                          void* ws, int accumulate, int* err, int cfg = 0);
// The two halves of syrk_tc_chunk: the fp16 slices of the chunk's rows, then the
// tensor-core kernel over them (timed on its own as the dominant kernel).
// corr (n2 doubles, or NULL) accumulates per row the part of the row's square
// sum that its fp16 slices do not represent (added to E'_aa by the finish).
cudaError_t syrk_tc_split(cudaStream_t st, const float2* B, int64_t sQ, int64_t sA, int64_t nJ, const int* qmap,
                          int64_t n2, int j0, int nq, const int* row_exp, void* split, double* corr);
cudaError_t syrk_tc_mma(cudaStream_t st, void* split, int64_t n2, int nq, int64_t nJ, const int2* tiles_d,
                        int ntiles, void* ws, int accumulate, int* err, int cfg);
// The finish fused with the chemist's permutation (eri: complex64 [p][q][r][s], or
// NULL; complex128 for the _z variant) and the FP64 traces of a Hermitian gamma
// (or NULL: out4 = E_J, E_K, 0, 0); part: syrk_tc_eri_part_count() double2 of
// scratch.  E is never stored.
size_t syrk_tc_eri_part_count();
cudaError_t syrk_tc_finish_eri(cudaStream_t st, const void* ws, int ntiles, const int* tile_of_d, const int2* orb,
                               int nf, const int* row_exp, const double* corr, double scale, float2* eri,
                               const double2* gamma, double2* part, double* out4);
cudaError_t syrk_tc_finish_eri_z(cudaStream_t st, const void* ws, int ntiles, const int* tile_of_d, const int2* orb,
                                 int nf, const int* row_exp, const double* corr, double scale, double2* eri,
                                 const double2* gamma, double2* part, double* out4);

// ---- FP64-class tensor-core contractions (k_tc64.cu): E' with four exact fp16
// slices of the float-float rows of B, B = M L with five exact slices of the
// float-float M and of L.  Same workspace, tile lists and finish as above.
size_t syrk4_tc_split_bytes(int64_t n2, int64_t kcols);
cudaError_t syrk4_tc_rowscale(cudaStream_t st, const ffcomplex* B, int64_t sQ, int64_t sA, int64_t nJ, int nS,
                              int64_t n2, int* row_exp);
cudaError_t syrk4_tc_split(cudaStream_t st, const ffcomplex* B, int64_t sQ, int64_t sA, int64_t nJ, int64_t n2,
                           int j0, int nq, const int* row_exp, void* split, double* corr);
cudaError_t syrk4_tc_mma(cudaStream_t st, void* split, int64_t n2, int nq, int64_t nJ, const int2* tiles_d,
                         int ntiles, void* ws, int accumulate, int* err);
int mlgemm5_tc_nj_pad(int nj);  // padded complex columns of B (multiple of 96)
int mlgemm5_tc_kp(int rp);
bool mlgemm5_tc_supported(int rp);
size_t mlgemm5_tc_lslice_bytes(int nk, int rp, int nj);
size_t mlgemm5_tc_split_bytes(int64_t n2, int rp, int nq);
cudaError_t mlgemm5_tc_prepare(cudaStream_t st, const double2* L, const double* sw, int nk, int np, const int* perm,
                               const int* rank, int rp, int nj, void* lsl, int* col_exp);
cudaError_t mlgemm5_tc_rowscale(cudaStream_t st, const ffcomplex* M, int64_t sq, int np, const int* qmap, int nS,
                                const int* perm, const int* rank, int rp, int64_t n2, int* row_exp);
cudaError_t mlgemm5_tc_chunk(cudaStream_t st, ffcomplex* M, int64_t sq, const int* qmap, int64_t n2, int np,
                             const int* perm, const int* rank, int rp, int nj, int j0, int nq, const int* row_exp,
                             void* split, const void* lsl, const int* col_exp, int nk, int* err);
// V_xi^q = Omega conj(c'^q) c'^q^T (Eq. 6) on the tensor cores, FP64-class: c' rows
// [q][I < rx][G < ng] float-float (q stride qs), V[q][I][J] complex128 (row pitch ldv,
// q stride vs).  work: vxi_tc_work_bytes(rx, ng, qc) bytes for chunks of qc q-points
// (vxi_tc_chunk picks qc for a byte budget); err: bounded-wait error word.
int vxi_tc_chunk(int rx, int ng, size_t budget);
size_t vxi_tc_work_bytes(int rx, int ng, int qc);
cudaError_t vxi_tc(cudaStream_t st, const ffcomplex* c, int64_t qs, int rx, int ng, int nq, double omega,
                   double2* V, int64_t ldv, int64_t vs, void* work, int qc, int* err);
// B^q = M^q L^q (w_q^{1/2} folded into L) on the tensor cores with three slices
// per operand (an integer and two fp16 remainders), over the structural nonzeros
// of L^q only: the rp = max_q r_q
// pivot columns perm_q[c] (c < rank_q) of M^q and the nj output columns.  M^q is
// stored by position j in the sum (q = qmap[j]) with q stride sq; B^q is written
// in place over it with row pitch nj.  prepare: slices of L for all q (once per
// L); rowscale: exponents of the gathered M rows over the sum; chunk: the
// positions j0..j0+nq-1 of the sum.
int mlgemm_tc_kp(int rp);
int mlgemm_tc_nj_pad(int nj);
bool mlgemm_tc_supported(int rp);
size_t mlgemm_tc_lslice_bytes(int nk, int rp, int nj);
size_t mlgemm_tc_split_bytes(int64_t n2, int rp, int nq);
cudaError_t mlgemm_tc_prepare(cudaStream_t st, const double2* L, const double* sw, int nk, int np, const int* perm,
                              const int* rank, int rp, int nj, void* lsl, int* col_exp);
cudaError_t mlgemm_tc_rowscale(cudaStream_t st, const float2* M, int64_t sq, int np, const int* qmap, int nS,
                               const int* perm, const int* rank, int rp, int64_t n2, int* row_exp);
cudaError_t mlgemm_tc_chunk(cudaStream_t st, float2* M, int64_t sq, const int* qmap, int64_t n2, int np,
                            const int* perm, const int* rank, int rp, int nj, int j0, int nq, const int* row_exp,
                            void* split, const void* lsl, const int* col_exp, int nk, int* err);
// eri[p][q][r][s] (complex64) = E[(p q)][(s r)] (complex128) * scale
cudaError_t eri_permute_zc(cudaStream_t st, const double2* E, int nf, double scale, float2* eri);

// E_ab += conj(E_{s(a)s(b)}), s((pq)) = (qp), in place (n_f^2 x n_f^2 complex128).
cudaError_t eri_swapconj_sym(cudaStream_t st, double2* E, int nf);
// out[b] = sw[b] L[b] over nb blocks of `per` elements (FP64 / to complex64).
cudaError_t scale_blocks(cudaStream_t st, const double2* L, int64_t per, int nb, const double* sw, double2* out);
cudaError_t scale_blocks_f(cudaStream_t st, const double2* L, int64_t per, int nb, const double* sw, float2* out);
// out[I][mu n_ao + nu] = conj(x1[I][mu]) x2[I][nu] for I < np (x1, x2: [np][n_ao]).
cudaError_t ao_pairs(cudaStream_t st, const double2* x1, const double2* x2, int np, int nao, double2* out);
// k-SOS-MP2 pieces: weighted orbital columns and the per-Q partial traces of
// the opposite-spin energy.
cudaError_t scale_cols(cudaStream_t st, const double2* y, int nk, int np, int nmo, int c0, int nc, const double* eps,
                       double sgn_tau, double2* out);
cudaError_t sos_trace_parts(cudaStream_t st, const double2* t, const double2* chi, const int kmesh[3], int np,
                            double* part);
// x[pairs[i].x] = conj(x[pairs[i].y]) for blocks of `per` elements (mirror_copy: plain copy).
cudaError_t mirror_conj(cudaStream_t st, double2* x, int64_t per, const int2* pairs, int npairs);
cudaError_t mirror_copy(cudaStream_t st, int32_t* x, int64_t per, const int2* pairs, int npairs);
// out[b][I][J] = a[b][J][I] * c[b][I][J] for nb blocks of n x n.
cudaError_t hadamard_t(cudaStream_t st, const double2* a, const double2* c, int n, int nb, double2* out);

// FP64-accurate complex GEMM on the tensor cores for 2K <= 128 (k_emu.cu):
// C_b = op(A_b) B_b, op 'N' or 'R' (conjugate), seven exact 7-bit slices per
// operand.  work: zgemm_emu_work_bytes(M, N, K, batch) bytes; err: device word
// set on a bounded-wait timeout.
bool zgemm_emu_supported(int K);
size_t zgemm_emu_work_bytes(int M, int N, int K, int batch);
cudaError_t zgemm_emu(cudaStream_t st, char opA, int M, int N, int K, const double2* A, int64_t lda, int64_t sA,
                      const double2* B, int64_t ldb, int64_t sB, double2* C, int64_t ldc, int64_t sC, int batch,
                      void* work, int* err);

// Precision conversions.
cudaError_t z2c(cudaStream_t st, const double2* in, float2* out, int64_t n);
cudaError_t c2z(cudaStream_t st, const float2* in, double2* out, int64_t n);

}  // namespace isdf
