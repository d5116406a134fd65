/*
 * isdf.h -- C ABI of the GB300 k-ISDF fragment-ERI library (libisdf.so).
 *
 * The library computes, on one GPU, the electron-repulsion integrals of
 * embedding / local-correlation fragments through translation-symmetry-adapted
 * interpolative separable density fitting (k-point FFTISDF).  The four steps
 * follow Section II of the paper:
 *
 *   isdf_build_points    Bloch GTOs on the grid (Eq. 1), interpolation points by
 *                        pivoted Cholesky of the pair products (Section II.A),
 *                        interpolating vectors X^k_{I mu} = phi^k_mu(r_I).
 *   isdf_fit_zeta        least-squares fit Pi^q xi^q = eta^q (Eqs. 2-5) with the
 *                        k-sums done as convolutions over the k-mesh (Algorithm 1).
 *   isdf_coulomb_metric  Coulomb kernel of the interpolation functions (Eq. 6) by
 *                        a grid FFT and a dense GEMM over G.
 *   isdf_fragment_eri    fragment ERIs (Eqs. 17-20, Algorithm 2):
 *                        (pq|rs) = (1/Nk) sum_q [M^q V^q M^q^H]_{(pq),(sr)} and the
 *                        Coulomb / exchange energy traces.
 *
 * Conventions shared by every call
 *   - Complex numbers are interleaved (re, im) doubles (complex128) unless a
 *     buffer is documented as complex64.  All arrays are row-major in the index
 *     order written next to them.
 *   - Grid: mesh n = (n0, n1, n2); point g has r = sum_i g_i/n_i a_i; flat index
 *     (g0*n1 + g1)*n2 + g2.  N_g = n0 n1 n2.
 *   - k-mesh: Gamma-centred, unfolded k = sum_i m_i/nk_i b_i, m_i in [0, nk_i),
 *     flat index (m0*nk1 + m1)*nk2 + m2.  q labels the same mesh.
 *   - The caller owns every buffer it passes; the handle owns all device
 *     workspaces (allocated on first use, reused on later calls, freed by
 *     isdf_destroy).  Device pointers must be on the handle's device.
 *   - All work is enqueued on the handle's CUDA stream.  A call returns after
 *     the host-visible outputs it writes are complete; device outputs are
 *     complete when the stream reaches the end of the call.
 *   - Every call returns an isdf_status; on failure isdf_last_error() holds a
 *     message.  No C++ exception crosses this boundary.  A handle is not
 *     thread-safe.
 */
#ifndef ISDF_H
#define ISDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct isdf_handle isdf_handle;

typedef enum {
  ISDF_OK = 0,
  ISDF_ERR_ARG = -1,      /* invalid argument (NULL, size, out-of-range value)   */
  ISDF_ERR_OOM = -2,      /* device allocation failed                             */
  ISDF_ERR_CUDA = -3,     /* a CUDA runtime call or kernel launch failed          */
  ISDF_ERR_NUMERIC = -4,  /* non-finite value, or a factorisation found rank 0 /  */
                          /* the point selection ran out of rank                 */
  ISDF_ERR_TIMEOUT = -5,  /* a bounded device-side wait expired                   */
  ISDF_ERR_STATE = -6     /* calls made out of order                              */
} isdf_status;

typedef enum {
  ISDF_FP64 = 0,   /* every step in FP64                                          */
  ISDF_MIXED = 1,  /* FP64-class points and fit (Eqs. 3-5); V (Eq. 6) from a float-  */
                   /* float grid FFT and V_xi on the tensor cores with four exact   */
                   /* fp16 slices; the fragment pair tensor and ERI contractions   */
                   /* (Eqs. 19-20) in reduced precision (FP32 transforms; fp16      */
                   /* integer + remainder slices on the tensor cores, ~2^-19 for E  */
                   /* and ~2^-30 for B = M L, relative)                             */
  ISDF_FP64_TC = 2 /* FP64-class results on the tensor cores: points and fit as in  */
                   /* ISDF_MIXED, V in FP64; the pair tensor in float-float (~2^-44), */
                   /* B = M L with five and E with four exact fp16 slices per       */
                   /* operand (~2^-28 of |R_a||R_b|; Ozaki-scheme emulation); the   */
                   /* ERIs complex128.  Falls back to FP64 arithmetic for a        */
                   /* fragment set whose 2 max r_q exceeds 576.                    */
} isdf_precision;

/* Cell, basis and sampling (Eq. 1; Section II).
 *   lattice     row i = lattice vector a_i in Bohr.
 *   coords      natm x 3 atom positions in Bohr.
 *   shells      Cartesian Gaussian shells: shell_atom[s], shell_l[s] (0..4),
 *               shell_nprim[s]; exps / coefs hold the primitives of all shells
 *               consecutively (coefs multiply *normalised* primitives).  AO order:
 *               shells in order, components x^lx y^ly z^lz with lx descending,
 *               then ly descending (s; x,y,z; xx,xy,xz,yy,yz,zz; ...).
 *   kmesh, mesh k-mesh and real-space grid per axis.
 *   lattice_eps lattice-sum truncation: images with alpha_min |r-T|^2 beyond
 *               -ln(lattice_eps) are dropped (0 selects exp(-40)).
 * The descriptor is copied by isdf_create; the caller may free it afterwards. */
typedef struct {
  double lattice[9];
  int natm;
  const double* coords;
  int nshell;
  const int* shell_atom;
  const int* shell_l;
  const int* shell_nprim;
  const double* exps;
  const double* coefs;
  int kmesh[3];
  int mesh[3];
  double lattice_eps;
} isdf_cell_desc;

/* Create a handle for `cell` computing in `precision`, enqueuing on
 * `cuda_stream` (a cudaStream_t; NULL = legacy default stream) of the current
 * device.  Limits: N_AO <= 1024, Nk <= 1024, nk_i <= 16, n_i <= 64. */
int isdf_create(const isdf_cell_desc* cell, isdf_precision precision, void* cuda_stream,
                isdf_handle** out);

/* Step S0-S1 (Eq. 1; Section II.A).  Evaluates phi^k_mu(r) on the grid and
 * selects n_p interpolation points by greedy pivoted Cholesky of the
 * pair-product Gram K(r,r') = |sum_k sum_mu conj(phi^k_mu(r)) phi^k_mu(r')|^2.
 * Residual diagonals within 1e-11 * d_max,0 of the largest (and at least half
 * of it) are ties, broken by the smallest splitmix64(seed ^ r).  Stops with
 * ISDF_ERR_NUMERIC if the largest residual falls below chol_tol * d_max,0
 * before n_p points are found.  ip_index_out: host int32[n_p] or NULL. */
int isdf_build_points(isdf_handle* h, int n_p, uint64_t seed, double chol_tol,
                      int32_t* ip_index_out);

/* Alternative to the selection: evaluate phi^k_mu(r) and take the n_p given
 * grid indices (host int32[n_p], each in [0, N_g), distinct) as the
 * interpolation points. */
int isdf_set_points(isdf_handle* h, int n_p, const int32_t* ip_index);

/* Step S2 (Eqs. 2-5, Algorithm 1).  Builds Pi^q and eta^q by convolutions over
 * the k-mesh, factorises Pi^q by pivoted Cholesky with relative truncation
 * solve_tol (pivot = largest remaining diagonal, ties to the smallest index;
 * dropped points get zeta = 0) and applies the factor to eta^q.
 * rank_out: host int32[Nk] (rank of each Pi^q) or NULL. */
int isdf_fit_zeta(isdf_handle* h, double solve_tol, int32_t* rank_out);

/* Step S3 (Eq. 6).  V^q_{IJ} = Omega sum_G conj(c^q_I(G)) c^q_J(G) 4 pi/|q+G|^2
 * with c^q_I(G) the normalised FFT of e^{-i q.r} zeta^q_I(r) and q+G = 0
 * dropped.  V_out: device complex128 [Nk][N_P][N_P], or NULL to keep V in the
 * handle only. */
int isdf_coulomb_metric(isdf_handle* h, void* V_out);

/* Step S3 by the route of Eqs. 7-8 (zeta never formed): V_eta^q from the grid
 * FFT of eta^q (Eq. 7, the integral of Eq. 6 with eta in place of zeta), then
 * the least-squares solution of Pi W Pi = V_eta (Eq. 8) through the same
 * truncated factor of Pi as isdf_fit_zeta: W^q = conj(Pi^+) V_eta conj(Pi^+)
 * (the conjugates express Eq. 8 in this library's index placement of Pi).
 * Produces the same V^q as isdf_coulomb_metric up to rounding, which here is
 * multiplied by cond(Pi^q) rather than its square root; computed in FP64 in
 * both precisions.  Replaces isdf_coulomb_metric (either may precede
 * isdf_fragment_eri).  V_out as for isdf_coulomb_metric. */
int isdf_coulomb_metric_eta(isdf_handle* h, void* V_out);

/* Step S4 (Eqs. 17-20, Algorithm 2).  For each fragment f with n_orb[f]
 * orbitals phi_p = Nk^{-1/2} sum_k sum_mu C^k_{mu p} phi^k_mu:
 *   C[f]       device complex128 [Nk][N_AO][n_orb[f]]
 *   gamma[f]   device complex128 [n_orb][n_orb] Hermitian density matrix with
 *              density n = sum_pq gamma_pq phi_p^* phi_q; array or entry may be NULL
 *   eri_out[f] complex128 [p][q][r][s] chemist's (pq|rs) in FP64 and FP64_TC
 *              mode, complex64 in MIXED mode; device memory or page-locked host
 *              memory (written by the kernel over the host link, e.g. when the
 *              ERIs of all fragments exceed HBM); array or entry may be NULL
 *   ej_out[f]  E_J = 1/2 sum gamma_pq gamma_rs (pq|rs)          (host, may be NULL)
 *   ek_out[f]  E_K = -1/4 sum gamma_ps gamma_rq (pq|rs)         (host, may be NULL)
 * The traces are accumulated in FP64.  Fragments are done one after the
 * other on the handle's stream (in MIXED mode small fragments are contracted
 * in groups, each fragment's results still written in turn), so several
 * entries of eri_out may name the same buffer (each result then overwrites the
 * previous one).
 * Device memory: the handle keeps its scratch between calls; when an
 * allocation for a fragment fails, the grid-sized fit arrays (eta, xi) are
 * freed and the allocation retried (isdf_get of eta or zeta and
 * isdf_coulomb_metric_eta then need a new isdf_fit_zeta); the fit frees the
 * fragment scratch in the same way. */
int isdf_fragment_eri(isdf_handle* h, int n_frag, const int32_t* n_orb,
                      const void* const* C, const void* const* gamma,
                      void* const* eri_out, double* ej_out, double* ek_out);

/* k-point exchange matrix from the ISDF integrals (Eq. 10), FP64:
 *   K^k_{mu nu} = -(1/Nk) sum_{k'} sum_{lam sig} P^{k'}_{lam sig} (mu k, lam k' | sig k', nu k)
 * computed as K^k = -(1/Nk) X^k^H Gamma^k X^k with
 *   rho^{k'} = X^{k'} P^{k'} X^{k'}^H  and  Gamma^k_IJ = sum_{k'} V^{k'-k}_JI rho^{k'}_IJ,
 * the k'-sum done as a convolution over the k-mesh (DFTs).
 *   P      device complex128 [Nk][N_AO][N_AO]: AO density matrix per k (density
 *          sum_k Phi^k_lam P^k_{lam sig} conj(Phi^k_sig) / Nk)
 *   K_out  device complex128 [Nk][N_AO][N_AO]
 * Needs the Coulomb metric (either route). */
int isdf_exchange(isdf_handle* h, const void* P, void* K_out);

/* Two-electron integrals of Bloch AOs for arbitrary k-quartets in the THC form
 * of Eq. 9, FP64, chemist's order:
 *   (mu k1 nu k2 | lam k3 sig k4)
 *     = Nk sum_IJ conj(X^{k1}_{I mu}) X^{k2}_{I nu} V^{Q}_{IJ} conj(X^{k3}_{J lam}) X^{k4}_{J sig},
 *   Q = k1 - k2,
 * for the Bloch AOs Phi^k_mu / sqrt(Nk) normalised over the Nk-cell supercell
 * (the fragment ERIs of isdf_fragment_eri for orbitals that are single Bloch
 * AOs).  The conjugates place the paper's X^{-k} = conj(X^k) on the first index
 * of each pair.
 *   quartets  host int32 [n_quartet][4]: flat k indices (k1, k2, k3, k4); every
 *             quartet must conserve crystal momentum, k1 - k2 = k4 - k3 on the
 *             mesh (other quartets vanish), else ISDF_ERR_ARG
 *   out       device complex128 [n_quartet][N_AO][N_AO][N_AO][N_AO]
 * Needs the Coulomb metric (either route). */
int isdf_ao_eri(isdf_handle* h, int n_quartet, const int32_t* quartets, void* out);

/* k-SOS-MP2 building blocks at one imaginary time tau >= 0 (Eqs. 11-15), FP64.
 * With orbital values at the points Y^k = X^k C^k and energies measured from a
 * chemical potential inside the gap:
 *   Go^k(tau) = Y_occ e^{+tau eps_i} Y_occ^H,   Gv^k(tau) = Y_vir e^{-tau eps_a} Y_vir^H,
 *   chi^Q_{IK}(tau) = sum_k Go^k_{KI}(tau) Gv^{k-Q}_{IK}(tau)      (P^Q = chi^Q V^Q),
 *   S(tau) = Nk^2 sum_Q tr[conj(V^Q) chi^Q conj(V^Q) (chi^{-Q})^T]
 *          = sum_{ia,jb} |(ia|jb)|^2 exp(-tau (eps_a - eps_i + eps_b - eps_j))
 * over the supercell, so that E_OS = -int_0^inf S(tau) dtau and
 * E_SOS-MP2 = 1.3 E_OS (Eq. 11).  The quadrature over tau is the caller's.
 * (The printed signs of Eq. 15 grow with tau; these are the decaying ones that
 * reproduce the Laplace form of the opposite-spin MP2 sum.)
 *   C        device complex128 [Nk][N_AO][n_mo] orbital coefficients per k
 *   eps      host double [Nk][n_mo] orbital energies; orbitals 0..n_occ-1 occupied
 *   chi_out  device complex128 [Nk][N_P][N_P], or NULL
 *   s_out    host double (S(tau)), or NULL
 * Needs the Coulomb metric (either route). */
int isdf_sos_polarizability(isdf_handle* h, const void* C, int n_mo, int n_occ, const double* eps, double tau,
                            void* chi_out, double* s_out);

/* Time-reversal pairing (default on).  The AO basis is real and the k-mesh
 * Gamma-centred, so Pi^{-q} = conj(Pi^q) and eta^{-q} = conj(eta^q) (Eqs. 4-5),
 * hence zeta^{-q} = conj(zeta^q) and V^{-q} = conj(V^q); and for any orbitals
 * M^{-q}_{(qp),I} = conj(M^q_{(pq),I}) (shift k by q in the k-sum of the pair
 * tensor, Eq. 20).  With pairing on:
 *   - isdf_fit_zeta and the Coulomb metric (both routes) compute the factor of
 *     Pi^q, xi^q and V^q only for q <= -q (index order) and set the others to
 *     the conjugates;
 *   - isdf_fragment_eri sums (pq|rs) = (1/Nk) sum_q [M^q V^q M^q^H] over about
 *     half of the q-points, since the term of -q is the term of q with the pair
 *     indices swapped and conjugated.
 * enable = 0 computes every q as written.  The results agree to rounding.
 * The setting applies to the calls made after it. */
int isdf_set_time_reversal(isdf_handle* h, int enable);

/* MIXED mode: device bytes that the fragment contraction may use for the fp16
 * slices of B (Algorithm 2's B^q = M^q L^q for all q).  B is sliced and
 * contracted in chunks of q-points that fit this limit, each chunk adding to
 * the same accumulator, so a smaller limit costs only more launches.  Default
 * 12 GiB; values below one q-point's slices give one q-point per chunk.
 * Returns ISDF_ERR_ARG for 0. */
int isdf_set_workspace_limit(isdf_handle* h, uint64_t bytes);

/* MIXED mode: schedule of the fragment contraction's tensor-core tiles.  The
 * lower-triangle tiles of E' are launched in bands of row blocks (the CTAs of
 * one wave then share their operand blocks in L2), by a kernel with one of two
 * pipelines (0: K rows of 64 fp16 in 3 stages; 1: rows of 32 fp16 in 6 stages).
 * With autotuning on (default), the first call that meets a tile list of a new
 * size class times its first q-chunk with the schedules (pipeline, band) =
 * (0, 12), (1, 12), (1, 6), (1, 24) and keeps the fastest for that class on this
 * handle; off, (0, 12) or the schedule fixed below is used.  The schedule
 * changes only the order of the
 * work, not the results.  isdf_autotune_report writes the choices as a JSON list
 * ([{"tiles": n, "pipeline": p, "band": b, "ms": [t0, t1, t2, t3]}, ...]) into
 * buf (len bytes, NUL-terminated; ISDF_ERR_ARG if it does not fit). */
int isdf_set_autotune(isdf_handle* h, int enable);
int isdf_autotune_report(const isdf_handle* h, char* buf, size_t len);
/* Fix the schedule instead of tuning it: pipeline 0 or 1 as above, band in
 * [1, 64] row blocks per band (turns autotuning off; isdf_set_autotune(h, 1)
 * turns it back on).  ISDF_ERR_ARG for other values. */
int isdf_set_tile_schedule(isdf_handle* h, int pipeline, int band);

/* Inspection of intermediate results (device outputs, complex128):
 *   what = 0  X   [Nk][N_P][N_AO]
 *   what = 1  Pi  [Nk][N_P][N_P]
 *   what = 2  eta [Nk][N_P][N_g]        (from isdf_fit_zeta until freed, see isdf_fragment_eri)
 *   what = 3  zeta [Nk][N_P][N_g]       (computed on request from the fit)
 * out must hold the whole array.  Returns ISDF_ERR_STATE if the step that
 * produces it has not run. */
int isdf_get(isdf_handle* h, int what, void* out);

/* Sizes: out[0]=N_AO, out[1]=Nk, out[2]=N_g, out[3]=N_P (0 before points). */
int isdf_sizes(const isdf_handle* h, int64_t* out);

/* Number of kernels this handle has launched since creation. */
int64_t isdf_launch_count(const isdf_handle* h);

/* Per-stage device timing with CUDA events recorded on the handle's stream.
 * isdf_timing_enable(h, 1) clears the totals and starts recording; 0 stops.
 * isdf_timing_get(h, stage, ...) returns, for
 *   stage 0  interpolation points (S0-S1)        stage 3  fragment pair tensor M^q (S4a)
 *   stage 1  fit of zeta (S2)                    stage 4  B^q = M^q L^q (S4b, first half)
 *   stage 2  Coulomb metric (S3)                 stage 5  E = sum_q B^q B^q^H (S4b, dominant)
 *   stage 6  the tensor-core kernel of stage 5 alone (mixed path: one record per
 *            launch of the E' kernel, without its slicing and finish)
 * the summed device milliseconds, the number of recorded launches of that
 * stage, and its algorithmic floating-point work (flops) summed over them. */
int isdf_timing_enable(isdf_handle* h, int enable);
int isdf_timing_get(const isdf_handle* h, int stage, double* ms_total, int64_t* launches,
                    double* flops_total);

/* Allocation-free variant of the fragment trace reduction.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device
 * memory -- for example a host application whose own allocator owns the GPU's
 * memory and forbids libraries to call cudaMalloc, or a latency-critical loop
 * that cannot afford the implicit synchronisation of an allocation.
 *   eri      device complex128 [p][q][r][s] chemist's (pq|rs) of one fragment
 *            (as written by isdf_fragment_eri in FP64 mode)
 *   gamma    device complex128 [n_orb][n_orb] density matrix (as above)
 *   ej_out, ek_out  host: E_J = 1/2 sum gamma_pq gamma_rs (pq|rs) and
 *            E_K = -1/4 sum gamma_ps gamma_rq (pq|rs), reduced in FP64
 *   cuda_stream     a cudaStream_t of the current device (NULL = default)
 * Needs no handle and allocates nothing: its scratch is a fixed 8 MiB array in
 * device global memory that every GPU loading the library holds until the
 * process exits.  Limit: n_orb <= 511; larger sizes return ISDF_ERR_ARG with
 * a message in isdf_last_error(NULL).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls share the array,
 * so calls that overlap on the GPU (other streams, other threads) race; the
 * call returns after the results are on the host. */
int isdf_eri_traces_noalloc(const void* eri, int n_orb, const void* gamma, double* ej_out, double* ek_out,
                            void* cuda_stream);

/* Message of the last failure: of the handle h, or (h == NULL) of the last
 * failed handle-free call on the calling thread. */
const char* isdf_last_error(const isdf_handle* h);
void isdf_destroy(isdf_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* ISDF_H */
