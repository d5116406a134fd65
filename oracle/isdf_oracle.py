"""Plain FP64 oracle of the k-ISDF fragment-ERI path (test infrastructure only).

This module is the slow, obviously-correct restatement of what the CUDA path
computes.  It is used only by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU baseline legs of ``bench.py``.  No product code imports it.

Conventions (all steps)
-----------------------
* Lattice rows ``a_i``; reciprocal rows ``b_i = 2 pi (A^{-1})^T``; cell volume
  Omega = |det A|.
* Grid point g = (g0, g1, g2), g_i in [0, n_i): r_g = sum_i g_i / n_i a_i; the
  flat index is row-major with the last axis fastest.
* Gamma-centred k-mesh, *not folded*: k_m = sum_i m_i / nk_i b_i with
  m_i in [0, nk_i); flat index row-major.  k +- q is taken mod nk_i per axis,
  which is exact because the Bloch AOs are periodic in k.
* G vectors follow fftfreq: h -> h if h < n/2 else h - n.
* Forward DFT carries exp(-i G.r); numpy.fft.fftn is used as that primitive.

Steps and the passages they follow
----------------------------------
* ``bloch_ao``       Eq. 1 (crystalline GTO as a lattice sum) on the FFTDF grid.
* ``select_ips``     Section II.A: interpolation points from a pivoted Cholesky
                     of the pair products phi^{k_mu}_mu(r) phi^{k_nu}_nu(r)^*
                     with r as the column index.
* ``metric_pi``      Eq. 4 (the metric Pi^q) via Eq. 3's least squares.
* ``rhs_eta``        Eq. 5 (the right-hand side eta^q).
* ``fit_zeta``       Eq. 3 (Pi^q xi^q = eta^q) solved by pivoted Cholesky.
* ``coulomb_metric`` Eq. 6 (Coulomb kernel of the interpolation functions).
* ``coulomb_metric_eta``  Eqs. 7-8 (the same kernel from eta, without zeta).
* ``fragment_T``, ``pair_tensor``  Eq. 20 and Algorithm 2 (the R^q intermediate).
* ``fragment_eri``   Eq. 19 (fragment ERIs from R^q and W^q).
* ``traces``         Coulomb / exchange energy traces of the fragment ERIs.
* ``exchange_matrix`` Eq. 10 (k-point exchange matrix from the ISDF integrals).

Readings of the paper used here (the paper is silent or ambiguous):
* The least-squares index placement of Eqs. 4-5 is taken as the normal
  equations of the fit of Eq. 2 with q = k_mu - k_nu (Section II.A); both
  placements give the same numbers because Pi^{-q} = conj(Pi^q).
* Algorithm 1's element-wise product is |T^R|^2 (T times its conjugate).
* Pi^q is factorised by a pivoted Cholesky with relative tolerance; dropped
  interpolation points get xi = 0 (basic solution).
* The q+G = 0 Coulomb term is dropped.
* Fragment orbitals are complex; the ERIs use the complex derivation that
  reduces to Eqs. 19-20 when C^{-k} = conj(C^k).
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import scipy.linalg as sla

__all__ = [
    "cart_exponents", "primitive_norm", "reciprocal", "grid_points", "grid_index_vectors",
    "kmesh_indices", "k_plus_table", "k_minus_table", "lattice_range", "ao_values",
    "bloch_ao", "splitmix64", "select_ips", "interp_vectors", "gram_k", "metric_pi",
    "g_values", "rhs_eta", "pchol", "pchol_solve", "fit_zeta", "gvectors_q",
    "coulomb_metric", "fragment_T", "pair_tensor", "fragment_E", "eri_from_E",
    "fragment_eri", "traces", "cheap_J", "run_isdf", "fftdf_fragment_eri",
    "supercell", "supercell_coefficients", "supercell_ips", "TIE_EPS", "LATTICE_EXP_CUT",
    "pinv_pchol", "coulomb_metric_eta", "exchange_matrix", "fftdf_exchange_matrix", "ao_eri",
    "green_ip", "polarizability", "sos_trace",
]

# exp(-40) tail rule of the lattice sum (Eq. 1): images whose Gaussian factor
# is below exp(-40) everywhere in the cell are outside the summation box.
LATTICE_EXP_CUT = 40.0
# Interpolation-point ties: residual diagonals within TIE_EPS * d_max,0 of the
# current maximum are equal candidates, broken by splitmix64(seed ^ r).
TIE_EPS = 1e-11


# ----------------------------------------------------------------------------
# Basis functions (Eq. 1)
# ----------------------------------------------------------------------------

def cart_exponents(l: int) -> List[Tuple[int, int, int]]:
    """Cartesian components of a shell: x before y before z (xx, xy, xz, yy, yz, zz)."""
    out = []
    for lx in range(l, -1, -1):
        for ly in range(l - lx, -1, -1):
            out.append((lx, ly, l - lx - ly))
    return out


def _dfact(n: int) -> float:
    """Double factorial with (-1)!! = 1."""
    r = 1.0
    while n > 1:
        r *= n
        n -= 2
    return r


def primitive_norm(alpha: float, lx: int, ly: int, lz: int) -> float:
    """N with integral of (N x^lx y^ly z^lz exp(-alpha r^2))^2 over R^3 equal to 1."""
    l = lx + ly + lz
    n2 = (2.0 * alpha / math.pi) ** 1.5 * (4.0 * alpha) ** l / (
        _dfact(2 * lx - 1) * _dfact(2 * ly - 1) * _dfact(2 * lz - 1))
    return math.sqrt(n2)


def reciprocal(lattice: np.ndarray) -> np.ndarray:
    """Rows b_i with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * math.pi * np.linalg.inv(lattice).T


def grid_index_vectors(mesh: Sequence[int]) -> np.ndarray:
    """(N_g, 3) integer grid indices in flat (row-major, last fastest) order."""
    g = np.indices(tuple(mesh)).reshape(3, -1).T
    return g.astype(np.int64)


def grid_points(cell) -> np.ndarray:
    """Cartesian coordinates of the uniform cell grid (Section II: FFTDF grid)."""
    g = grid_index_vectors(cell.mesh).astype(np.float64)
    frac = g / np.asarray(cell.mesh, dtype=np.float64)[None, :]
    return frac @ cell.lattice


def kmesh_indices(kmesh: Sequence[int]) -> np.ndarray:
    """(Nk, 3) integer m vectors of the Gamma-centred mesh, flat row-major order."""
    return np.indices(tuple(kmesh)).reshape(3, -1).T.astype(np.int64)


def _kflat(m: np.ndarray, kmesh: Sequence[int]) -> np.ndarray:
    km = np.asarray(kmesh)
    mm = np.mod(m, km)
    return (mm[..., 0] * km[1] + mm[..., 1]) * km[2] + mm[..., 2]


def k_plus_table(kmesh: Sequence[int]) -> np.ndarray:
    """kp[k, q] = flat index of k + q (mod the mesh)."""
    m = kmesh_indices(kmesh)
    return _kflat(m[:, None, :] + m[None, :, :], kmesh)


def k_minus_table(kmesh: Sequence[int]) -> np.ndarray:
    """km[k, q] = flat index of k - q (mod the mesh)."""
    m = kmesh_indices(kmesh)
    return _kflat(m[:, None, :] - m[None, :, :], kmesh)


def lattice_range(cell) -> np.ndarray:
    """Half-width L_i of the lattice-sum box |n_i| <= L_i (Eq. 1 truncation).

    R_cut = sqrt(40 / alpha_min); L_i = ceil(R_cut |b_i| / 2pi) + 1.
    """
    amin = min(min(s.exps) for s in cell.shells)
    rcut = math.sqrt(LATTICE_EXP_CUT / amin)
    b = reciprocal(cell.lattice)
    return np.array([int(math.ceil(rcut * np.linalg.norm(b[i]) / (2 * math.pi))) + 1 for i in range(3)])


def ao_values(cell, pts: np.ndarray) -> np.ndarray:
    """Real values of the reference-cell GTOs phi~_mu at the points: (N_AO, npts)."""
    out = []
    for sh in cell.shells:
        d = pts - cell.coords[sh.atom][None, :]
        r2 = np.einsum("ij,ij->i", d, d)
        for (lx, ly, lz) in cart_exponents(sh.l):
            radial = np.zeros(pts.shape[0])
            for a, c in zip(sh.exps, sh.coefs):
                radial += c * primitive_norm(a, lx, ly, lz) * np.exp(-a * r2)
            out.append(radial * d[:, 0] ** lx * d[:, 1] ** ly * d[:, 2] ** lz)
    return np.array(out)


def bloch_ao(cell, kidx: Optional[Sequence[int]] = None, pts: Optional[np.ndarray] = None) -> np.ndarray:
    """Crystalline GTOs on the grid, Eq. 1: Phi^k_mu(r) = sum_T e^{i k.T} phi~_mu(r - T).

    Returns (nk_sel, N_AO, npts) complex128 for the k-points `kidx` (all by default)
    at the points `pts` (the cell grid by default).  T runs over the full box
    |n_i| <= L_i of ``lattice_range``; e^{i k.T} = exp(2 pi i sum_i m_i n_i / nk_i).
    """
    if pts is None:
        pts = grid_points(cell)
    m = kmesh_indices(cell.kmesh)
    if kidx is not None:
        m = m[np.asarray(kidx)]
    L = lattice_range(cell)
    nk_arr = np.asarray(cell.kmesh, dtype=np.float64)
    phi = np.zeros((m.shape[0], cell.nao, pts.shape[0]), np.complex128)
    for n0 in range(-L[0], L[0] + 1):
        for n1 in range(-L[1], L[1] + 1):
            for n2 in range(-L[2], L[2] + 1):
                n = np.array([n0, n1, n2])
                T = n @ cell.lattice
                v = ao_values(cell, pts - T[None, :])
                phase = np.exp(2j * math.pi * (m @ (n / nk_arr)))
                phi += phase[:, None, None] * v[None, :, :]
    return phi


# ----------------------------------------------------------------------------
# Interpolation points (Section II.A, pivoted Cholesky of the pair products)
# ----------------------------------------------------------------------------

_M64 = (1 << 64) - 1


def splitmix64(x) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea & Flood 2014), elementwise on uint64."""
    z = np.asarray(x, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def select_ips(phi: np.ndarray, n_p: int, seed: int, chol_tol: float = 1e-14,
               tie_eps: float = TIE_EPS) -> Tuple[np.ndarray, int]:
    """Greedy pivoted Cholesky of the pair-product Gram over grid points.

    The pair products rho^{k1 k2}_{mu nu}(r) = Phi^{k1}_mu(r) conj(Phi^{k2}_nu(r))
    with r as column index have the Gram matrix
        K(r, r') = sum_{pairs} conj(rho(r)) rho(r') = |D(r, r')|^2,
        D(r, r') = sum_k sum_mu conj(Phi^k_mu(r)) Phi^k_mu(r').
    The largest-residual columns are taken one at a time (textbook pivoted
    Cholesky, columns of K generated on demand).  Ties: all unchosen r with
    d_r >= d_max - tie_eps * d_max,0 and d_r >= d_max / 2 are candidates and
    the one with the smallest splitmix64(seed ^ r) wins.  Stops early when the
    largest residual falls below chol_tol * d_max,0.

    Returns (ips, n_found).
    """
    nk, nao, ng = phi.shape
    F = phi.reshape(nk * nao, ng)
    Ddiag = np.sum(np.abs(F) ** 2, axis=0)
    d = Ddiag ** 2
    d0 = float(d.max())
    chosen = np.zeros(ng, bool)
    Lmat = np.zeros((ng, n_p))
    hashes = splitmix64(np.uint64(seed) ^ np.arange(ng, dtype=np.uint64))
    ips = []
    for j in range(n_p):
        dm = np.where(chosen, -np.inf, d)
        dmax = float(dm.max())
        if not (dmax >= chol_tol * d0) or dmax <= 0.0:
            break
        cand = np.nonzero((dm >= dmax - tie_eps * d0) & (dm >= 0.5 * dmax))[0]
        p = int(cand[np.argmin(hashes[cand])])
        Dcol = F.conj().T @ F[:, p]
        Kcol = np.abs(Dcol) ** 2
        l = (Kcol - Lmat[:, :j] @ Lmat[p, :j]) / math.sqrt(d[p])
        Lmat[:, j] = l
        d = d - l * l
        chosen[p] = True
        ips.append(p)
    return np.array(ips, dtype=np.int64), len(ips)


def interp_vectors(phi: np.ndarray, ips: np.ndarray) -> np.ndarray:
    """Interpolating vectors X^k_{I mu} = phi^k_mu(r_I) (text after Eq. 2): (Nk, N_P, N_AO)."""
    return np.ascontiguousarray(phi[:, :, ips].transpose(0, 2, 1))


# ----------------------------------------------------------------------------
# Least-squares fit (Eqs. 2-5)
# ----------------------------------------------------------------------------

def gram_k(X: np.ndarray) -> np.ndarray:
    """G^k_{IJ} = sum_mu conj(X^k_{I mu}) X^k_{J mu}: (Nk, N_P, N_P)."""
    return np.einsum("kim,kjm->kij", X.conj(), X)


def metric_pi(X: np.ndarray, kmesh: Sequence[int], qs: Optional[Sequence[int]] = None) -> np.ndarray:
    """Metric of the normal equations, Eq. 4, by the direct k-sum.

    For the fit of pairs Phi^k_mu conj(Phi^{k-q}_nu) (momentum q) the metric is
    Pi^q_{IJ} = sum_k sum_{mu nu} conj(X^k_{I mu} conj(X^{k-q}_{I nu})) X^k_{J mu} conj(X^{k-q}_{J nu})
              = sum_k G^k_{IJ} conj(G^{k-q}_{IJ}).
    """
    G = gram_k(X)
    km = k_minus_table(kmesh)
    nk = X.shape[0]
    qs = range(nk) if qs is None else qs
    out = []
    for q in qs:
        acc = np.zeros(G.shape[1:], np.complex128)
        for k in range(nk):
            acc += G[k] * G[km[k, q]].conj()
        out.append(acc)
    return np.array(out)


def g_values(X: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """g^k_I(r) = sum_mu conj(X^k_{I mu}) Phi^k_mu(r): (Nk, N_P, npts)."""
    return np.einsum("kim,kmr->kir", X.conj(), phi)


def rhs_eta(X: np.ndarray, phi: np.ndarray, kmesh: Sequence[int],
            qs: Optional[Sequence[int]] = None, g: Optional[np.ndarray] = None) -> np.ndarray:
    """Right-hand side, Eq. 5, by the direct k-sum:
    eta^q_I(r) = sum_k g^k_I(r) conj(g^{k-q}_I(r))."""
    if g is None:
        g = g_values(X, phi)
    km = k_minus_table(kmesh)
    nk = X.shape[0]
    qs = range(nk) if qs is None else qs
    out = []
    for q in qs:
        acc = np.zeros(g.shape[1:], np.complex128)
        for k in range(nk):
            acc += g[k] * g[km[k, q]].conj()
        out.append(acc)
    return np.array(out)


def pchol(A: np.ndarray, tol: float, tie_eps: float = TIE_EPS) -> Tuple[np.ndarray, np.ndarray, int]:
    """Pivoted Cholesky of a Hermitian PSD matrix, A ~ L L^H (textbook, right-looking).

    Pivot = largest remaining diagonal; diagonals within tie_eps * d_max,0 of it
    (and at least half of it) are ties, resolved to the smallest index.  Stops
    when the largest remaining diagonal is <= tol * d_max,0.  Returns
    (L, perm, rank) with L of shape (n, rank) and perm the pivot order.
    """
    n = A.shape[0]
    d = np.real(np.diagonal(A)).astype(np.float64).copy()
    dmax0 = float(d.max()) if n else 0.0
    L = np.zeros((n, n), A.dtype)
    perm: List[int] = []
    used = np.zeros(n, bool)
    for j in range(n):
        dm = np.where(used, -np.inf, d)
        dmax = float(dm.max())
        if not (dmax > tol * dmax0) or dmax <= 0.0:
            break
        thr = max(dmax - tie_eps * dmax0, 0.5 * dmax)
        p = int(np.nonzero(dm >= thr)[0][0])
        col = A[:, p] - L[:, :j] @ L[p, :j].conj()
        L[:, j] = col / math.sqrt(dm[p])
        d = d - np.abs(L[:, j]) ** 2
        used[p] = True
        perm.append(p)
    r = len(perm)
    return L[:, :r], np.array(perm, dtype=np.int64), r


def pchol_solve(L: np.ndarray, perm: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Basic solution of A x = B from the pivoted factor: rows outside perm are 0."""
    r = len(perm)
    x = np.zeros((L.shape[0],) + B.shape[1:], np.result_type(L, B))
    if r == 0:
        return x
    Ls = L[perm, :r]                       # lower triangular in pivot order
    y = sla.solve_triangular(Ls, B[perm], lower=True)
    x[perm] = sla.solve_triangular(Ls.conj().T, y, lower=False)
    return x


def fit_zeta(Pi: np.ndarray, eta: np.ndarray, solve_tol: float) -> Tuple[np.ndarray, np.ndarray]:
    """Eq. 3 per q: Pi^q zeta^q = eta^q.  Returns (zeta, rank per q)."""
    zeta = np.zeros_like(eta)
    ranks = np.zeros(Pi.shape[0], np.int64)
    for i in range(Pi.shape[0]):
        L, perm, r = pchol(Pi[i], solve_tol)
        zeta[i] = pchol_solve(L, perm, eta[i])
        ranks[i] = r
    return zeta, ranks


# ----------------------------------------------------------------------------
# Coulomb kernel (Eq. 6)
# ----------------------------------------------------------------------------

def gvectors_q(cell, q: int) -> np.ndarray:
    """Cartesian q + G for every FFT index of the cell grid (fftfreq G), (N_g, 3)."""
    mq = kmesh_indices(cell.kmesh)[q].astype(np.float64)
    h = grid_index_vectors(cell.mesh)
    mesh = np.asarray(cell.mesh)
    ghat = np.where(h < mesh[None, :] / 2.0, h, h - mesh[None, :]).astype(np.float64)
    frac = mq[None, :] / np.asarray(cell.kmesh, np.float64)[None, :] + ghat
    return frac @ reciprocal(cell.lattice)


def coulomb_metric(cell, zeta: np.ndarray, qs: Sequence[int]) -> np.ndarray:
    """Eq. 6 for each q in qs (zeta[i] belongs to qs[i]):

    u^q_I(r) = e^{-i q.r} zeta^q_I(r) (cell periodic),  c^q_I(G) = N_g^{-1} sum_r u e^{-i G.r},
    V^q_{IJ} = Omega sum_G conj(c^q_I(G)) c^q_J(G) 4 pi / |q+G|^2,  q+G = 0 dropped.
    """
    mesh = tuple(cell.mesh)
    ng = cell.ngrid
    gi = grid_index_vectors(mesh).astype(np.float64)
    mk = kmesh_indices(cell.kmesh).astype(np.float64)
    out = []
    for i, q in enumerate(qs):
        ang = np.sum(mk[q][None, :] * gi / (np.asarray(cell.kmesh, np.float64) * np.asarray(mesh, np.float64))[None, :], axis=1)
        u = zeta[i] * np.exp(-2j * math.pi * ang)[None, :]
        c = np.fft.fftn(u.reshape((-1,) + mesh), axes=(1, 2, 3)).reshape(u.shape[0], ng) / ng
        qg = gvectors_q(cell, q)
        g2 = np.einsum("ij,ij->i", qg, qg)
        w = np.zeros(ng)
        nz = g2 > 1e-300
        w[nz] = 4.0 * math.pi / g2[nz]
        out.append(cell.volume * (c.conj() * w[None, :]) @ c.T)
    return np.array(out)


def pinv_pchol(A: np.ndarray, tol: float) -> np.ndarray:
    """Basic pseudo-inverse from the pivoted Cholesky: A^+ = P_S (A_SS)^{-1} P_S^T,
    zero outside the kept pivots S (the same truncation as the solve of Eq. 3)."""
    L, perm, r = pchol(A, tol)
    out = np.zeros_like(A)
    if r:
        Ls = L[perm, :r]
        inv = sla.solve_triangular(Ls, np.eye(r, dtype=A.dtype), lower=True)
        out[np.ix_(perm, perm)] = inv.conj().T @ inv
    return out


def coulomb_metric_eta(cell, Pi: np.ndarray, eta: np.ndarray, solve_tol: float,
                       qs: Optional[Sequence[int]] = None) -> np.ndarray:
    """Coulomb kernel without forming zeta (Eqs. 7-8): V^q from the fitting
    right-hand side eta^q (Eq. 7, the same integral as Eq. 6 with eta in place of
    xi), then the least-squares solution of Pi W Pi = V (Eq. 8) through the
    truncated pseudo-inverse of the solve: W = conj(Pi^+) V conj(Pi^+).  The
    conjugates follow from zeta = Pi^+ eta with the Hermitian Pi of Eq. 4 in the
    index placement used here (Eq. 8 reads Pi^T W Pi^T = V in that placement)."""
    nk = Pi.shape[0]
    qs = list(range(nk)) if qs is None else list(qs)
    Veta = coulomb_metric(cell, eta, qs)
    out = []
    for i, q in enumerate(qs):
        P = pinv_pchol(Pi[q], solve_tol).conj()
        out.append(P @ Veta[i] @ P)
    return np.array(out)


# ----------------------------------------------------------------------------
# Fragment ERIs (Eqs. 17-20, Algorithm 2)
# ----------------------------------------------------------------------------

def fragment_T(X: np.ndarray, C: np.ndarray) -> np.ndarray:
    """T^k_{Ip} = sum_mu X^k_{I mu} C^k_{mu p}: (Nk, N_P, n_f)."""
    return np.einsum("kim,kmp->kip", X, C)


def pair_tensor(T: np.ndarray, kmesh: Sequence[int], qs: Optional[Sequence[int]] = None) -> np.ndarray:
    """Fragment pair tensor by the direct k-sum (Eq. 20 in complex form):

    M^Q_{(pq), I} = sum_k T^k_{Iq} conj(T^{k+Q}_{Ip}),  shape (nQ, n_f*n_f, N_P).
    """
    kp = k_plus_table(kmesh)
    nk, npt, nf = T.shape
    qs = range(nk) if qs is None else qs
    out = []
    for Q in qs:
        acc = np.zeros((nf, nf, npt), np.complex128)
        for k in range(nk):
            acc += np.einsum("ip,iq->pqi", T[kp[k, Q]].conj(), T[k])
        out.append(acc.reshape(nf * nf, npt))
    return np.array(out)


def fragment_E(M: np.ndarray, V: np.ndarray, nk: int) -> np.ndarray:
    """E = (1/Nk) sum_Q M^Q V^Q M^Q^H over the Q in the arrays (Eq. 19)."""
    E = np.zeros((M.shape[1], M.shape[1]), np.complex128)
    for i in range(M.shape[0]):
        E += M[i] @ V[i] @ M[i].conj().T
    return E / nk


def eri_from_E(E: np.ndarray, nf: int) -> np.ndarray:
    """Chemist's (pq|rs) = E_{(pq),(sr)}: returns the [p][q][r][s] array."""
    return np.ascontiguousarray(E.reshape(nf, nf, nf, nf).transpose(0, 1, 3, 2))


def fragment_eri(X: np.ndarray, V: np.ndarray, C: np.ndarray, kmesh: Sequence[int]) -> np.ndarray:
    """Fragment ERIs (pq|rs) over all Q (Eqs. 19-20)."""
    T = fragment_T(X, C)
    M = pair_tensor(T, kmesh)
    return eri_from_E(fragment_E(M, V, X.shape[0]), C.shape[2])


def traces(eri: np.ndarray, gamma: np.ndarray) -> Tuple[float, float]:
    """E_J = 1/2 sum gamma_pq gamma_rs (pq|rs);  E_K = -1/4 sum gamma_ps gamma_rq (pq|rs).

    Closed-shell, spin-summed gamma with density n = sum_pq gamma_pq phi_p^* phi_q.
    """
    ej = 0.5 * np.einsum("pq,rs,pqrs->", gamma, gamma, eri)
    ek = -0.25 * np.einsum("ps,rq,pqrs->", gamma, gamma, eri)
    return float(ej.real), float(ek.real)


def cheap_J(M: np.ndarray, V: np.ndarray, gamma: np.ndarray, nk: int) -> float:
    """E_J without the ERIs: a^Q_I = sum_pq gamma_pq M^Q_{(pq),I};
    E_J = 1/(2 Nk) sum_Q a^Q V^Q conj(a^Q)."""
    g = gamma.reshape(-1)
    tot = 0.0 + 0.0j
    for i in range(M.shape[0]):
        a = g @ M[i]
        tot += a @ V[i] @ a.conj()
    return float((tot / (2.0 * nk)).real)


# ----------------------------------------------------------------------------
# AO-level integrals for arbitrary k-quartets (Eq. 9)
# ----------------------------------------------------------------------------

def ao_eri(X: np.ndarray, V: np.ndarray, quartets: Sequence[Sequence[int]], kmesh: Sequence[int]) -> np.ndarray:
    """(mu k1 nu k2 | lam k3 sig k4) of the Bloch AOs Phi^k / sqrt(Nk) (normalised
    over the Nk-cell supercell), chemist's order, from the ISDF factors (Eq. 9):

      Nk sum_IJ conj(X^{k1}_{I mu}) X^{k2}_{I nu} V^{Q}_{IJ} conj(X^{k3}_{J lam}) X^{k4}_{J sig},
      Q = k1 - k2, which must equal k4 - k3 (crystal momentum; other quartets vanish).

    Written directly from the definition of the fragment ERIs for orbitals that are
    single Bloch AOs.  Returns (n_quartets, N_AO, N_AO, N_AO, N_AO)."""
    nk = X.shape[0]
    km = k_minus_table(kmesh)
    kp = k_plus_table(kmesh)
    out = []
    for k1, k2, k3, k4 in quartets:
        Q = km[k1, k2]                      # k1 - k2
        if kp[k3, Q] != k4:                 # k4 = k3 + Q
            raise ValueError("quartet does not conserve crystal momentum")
        A = np.einsum("im,in->imn", X[k1].conj(), X[k2])     # (N_P, mu, nu)
        Cc = np.einsum("jl,js->jls", X[k3].conj(), X[k4])    # (N_P, lam, sig)
        out.append(nk * np.einsum("imn,ij,jls->mnls", A, V[Q], Cc))
    return np.array(out)


# ----------------------------------------------------------------------------
# k-SOS-MP2 polarisability in the interpolation-point basis (Eqs. 11-15)
# ----------------------------------------------------------------------------

def green_ip(X: np.ndarray, C: np.ndarray, eps: np.ndarray, n_occ: int, tau: float) -> Tuple[np.ndarray, np.ndarray]:
    """Imaginary-time Green's functions of the occupied and the virtual orbitals at
    the interpolation points, for tau >= 0 (Eq. 15 with decaying exponentials):

      Go^k_{IJ}(tau) = sum_{i occ} Y^k_{Ii} conj(Y^k_{Ji}) exp(+tau eps^k_i),
      Gv^k_{IJ}(tau) = sum_{a vir} Y^k_{Ia} conj(Y^k_{Ja}) exp(-tau eps^k_a),
      Y^k = X^k C^k  (orbital values at the points, Eq. 14),

    with energies measured from a chemical potential inside the gap."""
    Y = np.einsum("kim,kmn->kin", X, C)
    wo = np.exp(tau * eps[:, :n_occ])
    wv = np.exp(-tau * eps[:, n_occ:])
    Go = np.einsum("kin,kn,kjn->kij", Y[:, :, :n_occ], wo, Y[:, :, :n_occ].conj())
    Gv = np.einsum("kia,ka,kja->kij", Y[:, :, n_occ:], wv, Y[:, :, n_occ:].conj())
    return Go, Gv


def polarizability(Go: np.ndarray, Gv: np.ndarray, kmesh: Sequence[int]) -> np.ndarray:
    """chi^Q_{IK}(tau) = sum_k Go^k_{KI}(tau) Gv^{k-Q}_{IK}(tau)  (Eq. 13 before the
    kernel: the element-wise k-convolution of the two Green's functions), by the
    direct k-sum.  chi^Q is Hermitian positive semidefinite."""
    km = k_minus_table(kmesh)
    nk = Go.shape[0]
    out = np.zeros_like(Go)
    for Q in range(nk):
        for k in range(nk):
            out[Q] += Go[k].T * Gv[km[k, Q]]
    return out


def sos_trace(chi: np.ndarray, V: np.ndarray, kmesh: Sequence[int]) -> float:
    """S(tau) = Nk^2 sum_Q tr[conj(V^Q) chi^Q conj(V^Q) (chi^{-Q})^T] = sum_{ia,jb}
    |(ia|jb)|^2 exp(-tau (eps_a - eps_i + eps_b - eps_j)) over the orbitals of the
    Nk-cell supercell (Eq. 12 with P^Q = chi^Q V^Q).  The opposite-spin energy of
    the supercell is E_OS = -int_0^inf S(tau) dtau, and E_SOS-MP2 = 1.3 E_OS (Eq. 11)."""
    nk = chi.shape[0]
    km = k_minus_table(kmesh)
    tot = 0.0 + 0.0j
    for Q in range(nk):
        Vc = V[Q].conj()
        tot += np.trace(Vc @ chi[Q] @ Vc @ chi[km[0, Q]].T)
    return float((nk * nk * tot).real)


# ----------------------------------------------------------------------------
# k-point exchange matrix (Eq. 10)
# ----------------------------------------------------------------------------

def exchange_matrix(X: np.ndarray, V: np.ndarray, P: np.ndarray, kmesh: Sequence[int]) -> np.ndarray:
    """K^k_{mu nu} = -(1/Nk) sum_{k'} sum_{lam sig} P^{k'}_{lam sig} (mu k, lam k' | sig k', nu k)
    with the ISDF integrals (Eq. 9), by the direct k-sum of Eq. 10:

      rho^{k'}_{IJ} = sum_{lam sig} X^{k'}_{I lam} P^{k'}_{lam sig} conj(X^{k'}_{J sig}),
      Gamma^k_{IJ}  = sum_{k'} V^{k'-k}_{JI} rho^{k'}_{IJ},
      K^k = -(1/Nk) X^k^H Gamma^k X^k.

    P is the AO density matrix per k with the density sum_{k lam sig}
    Phi^k_lam(r) P^k_{lam sig} conj(Phi^k_sig(r)) / Nk."""
    nk = X.shape[0]
    km = k_minus_table(kmesh)
    rho = np.einsum("kil,kls,kjs->kij", X, P, X.conj())
    out = []
    for k in range(nk):
        G = np.zeros(rho.shape[1:], np.complex128)
        for kp in range(nk):
            G += V[km[kp, k]].T * rho[kp]
        out.append(-(X[k].conj().T @ G @ X[k]) / nk)
    return np.array(out)


def fftdf_exchange_matrix(cell, P: np.ndarray, phi: Optional[np.ndarray] = None) -> np.ndarray:
    """Grid-exact exchange (no density fitting): for each k, k' the pair densities
    conj(Phi^k_mu) Phi^{k'}_lam (momentum k' - k) are Poisson-solved on the cell grid
    with the weights 4 pi/|q+G|^2 (q+G = 0 dropped) and contracted as in Eq. 10."""
    if phi is None:
        phi = bloch_ao(cell)
    nk, nao, ng = phi.shape
    km = k_minus_table(cell.kmesh)
    mesh = tuple(cell.mesh)
    gi = grid_index_vectors(mesh).astype(np.float64)
    mk = kmesh_indices(cell.kmesh).astype(np.float64)
    den = (np.asarray(cell.kmesh, np.float64) * np.asarray(mesh, np.float64))[None, :]
    K = np.zeros((nk, nao, nao), np.complex128)
    for k in range(nk):
        for kp in range(nk):
            q = km[kp, k]
            # rho_{mu lam}(r) = conj(Phi^k_mu) Phi^{k'}_lam, Bloch with momentum q = k' - k
            rho = (phi[k].conj()[:, None, :] * phi[kp][None, :, :]).reshape(nao * nao, ng)
            u = rho * np.exp(-2j * math.pi * np.sum(mk[q][None, :] * gi / den, axis=1))[None, :]
            c = np.fft.fftn(u.reshape((-1,) + mesh), axes=(1, 2, 3)).reshape(nao * nao, ng) / ng
            qg = gvectors_q(cell, q)
            g2 = np.einsum("ij,ij->i", qg, qg)
            w = np.zeros(ng)
            nz = g2 > 1e-300
            w[nz] = 4.0 * math.pi / g2[nz]
            # V4[mu][lam][nu][sig] = int conj(rho_{mu lam}) v rho_{nu sig}; the second density of
            # (mu k lam k' | sig k' nu k) is conj(rho_{nu sig}), so that integral is conj(V4)
            Vmat = cell.volume * (c.conj() * w[None, :]) @ c.T
            V4 = Vmat.reshape(nao, nao, nao, nao)
            K[k] += -np.einsum("ls,mlns->mn", P[kp], V4.conj()) / nk
    return K

# ----------------------------------------------------------------------------
# Whole path
# ----------------------------------------------------------------------------

def run_isdf(cell, n_p: int, seed: int, chol_tol: float = 1e-14, solve_tol: float = 1e-12,
             ips: Optional[np.ndarray] = None, phi: Optional[np.ndarray] = None) -> Dict[str, np.ndarray]:
    """Steps S0-S3 for all q: Phi, IPs, X, Pi, eta, zeta, V."""
    if phi is None:
        phi = bloch_ao(cell)
    if ips is None:
        ips, nfound = select_ips(phi, n_p, seed, chol_tol)
        if nfound < n_p:
            raise RuntimeError(f"pivoted Cholesky stopped after {nfound} of {n_p} points")
    X = interp_vectors(phi, ips)
    nk = cell.nkpts
    Pi = metric_pi(X, cell.kmesh)
    eta = rhs_eta(X, phi, cell.kmesh)
    zeta, ranks = fit_zeta(Pi, eta, solve_tol)
    V = coulomb_metric(cell, zeta, range(nk))
    return dict(phi=phi, ips=ips, X=X, Pi=Pi, eta=eta, zeta=zeta, ranks=ranks, V=V)


# ----------------------------------------------------------------------------
# Pin helpers: grid-exact ERIs and the Gamma-point supercell
# ----------------------------------------------------------------------------

def supercell(cell):
    """The Nk-image Gamma-point supercell of `cell` (images R in [0, nk)^3)."""
    from paper_2601_16379_gb300.workloads import Cell, Shell
    km = np.asarray(cell.kmesh)
    Rs = kmesh_indices(cell.kmesh)
    natm = cell.coords.shape[0]
    coords = []
    shells = []
    for iR, R in enumerate(Rs):
        shift = R @ cell.lattice
        for a in range(natm):
            coords.append(cell.coords[a] + shift)
        for s in cell.shells:
            shells.append(Shell(iR * natm + s.atom, s.l, s.exps, s.coefs))
    lat = cell.lattice * km[:, None]
    mesh = tuple(int(x) for x in np.asarray(cell.mesh) * km)
    return Cell(lat, np.array(coords), shells, (1, 1, 1), mesh)


def supercell_coefficients(cell, C: np.ndarray) -> np.ndarray:
    """C^Gamma_{(R mu), p} = Nk^{-1/2} sum_k C^k_{mu p} e^{i k.R}: (1, Nk*N_AO, n_f)."""
    m = kmesh_indices(cell.kmesh).astype(np.float64)
    nk_arr = np.asarray(cell.kmesh, np.float64)
    ph = np.exp(2j * math.pi * (m / nk_arr[None, :]) @ m.T)   # [k, R] = e^{i k.R}
    CR = np.einsum("kR,kmp->Rmp", ph, C) / math.sqrt(C.shape[0])
    return CR.reshape(1, -1, C.shape[2])


def supercell_ips(cell, ips: np.ndarray) -> np.ndarray:
    """Flat supercell-grid indices of the translated images r_I + R."""
    mesh = np.asarray(cell.mesh)
    km = np.asarray(cell.kmesh)
    big = mesh * km
    g = grid_index_vectors(cell.mesh)[ips]
    out = []
    for R in kmesh_indices(cell.kmesh):
        gg = g + (R * mesh)[None, :]
        out.append((gg[:, 0] * big[1] + gg[:, 1]) * big[2] + gg[:, 2])
    return np.concatenate(out)


def fftdf_fragment_eri(cell, C: np.ndarray) -> np.ndarray:
    """Grid-exact fragment ERIs on the supercell grid (no density fitting).

    phi_p(r + R) = Nk^{-1/2} sum_k sum_mu C^k_{mu p} e^{i k.R} Phi^k_mu(r);
    (pq|rs) = Omega_sc sum_K conj(rhohat_qp(K)) rhohat_rs(K) 4 pi / |K|^2 with
    rho_pq = conj(phi_p) phi_q, rhohat = DFT / N_sc, fftfreq K of the supercell, K = 0 dropped.
    """
    sc = supercell(cell)
    CG = supercell_coefficients(cell, C)
    phiG = bloch_ao(sc)[0]                     # (Nk*N_AO, N_sc), real up to rounding
    orb = CG[0].T @ phiG                       # (n_f, N_sc)
    nf = orb.shape[0]
    nsc = sc.ngrid
    rho = (orb.conj()[:, None, :] * orb[None, :, :]).reshape(nf * nf, nsc)
    rhat = np.fft.fftn(rho.reshape((-1,) + sc.mesh), axes=(1, 2, 3)).reshape(nf * nf, nsc) / nsc
    K = gvectors_q(sc, 0)
    k2 = np.einsum("ij,ij->i", K, K)
    w = np.zeros(nsc)
    nz = k2 > 1e-300
    w[nz] = 4.0 * math.pi / k2[nz]
    # H_{(ab),(cd)} = Omega_sc sum_K conj(rhohat_ab) w rhohat_cd = (ba|cd)
    H = sc.volume * (rhat.conj() * w[None, :]) @ rhat.T
    H4 = H.reshape(nf, nf, nf, nf)             # [a][b][c][d] = (b a | c d)
    return np.ascontiguousarray(H4.transpose(1, 0, 2, 3))
