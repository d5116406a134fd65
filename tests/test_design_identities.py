"""Identities the GPU path is built on, checked in FP64 on the oracle's arrays.

The fragment contraction on the GPU does not form E = sum_q M^q V^q M^q^H as
written (Eq. 19).  It relies on two exact rewritings, which these CPU tests
check on the oracle's pair tensor and Coulomb metric:

* the structural zeros of L^q (V^q = L^q L^q^H with L^q = W^T L_xi): L^q is
  nonzero only in the pivot rows of the truncated factor of Pi^q and in the
  columns below the rank of V_xi, so B^q = M^q L^q needs only those;
* the real symmetric form: in the basis u = e_(pq) + e_(qp), v = i (e_(pq) - e_(qp)),
  e_(pp) fixed by the time-reversal symmetry E_{s(a)s(b)} = conj(E_ab), E is real,
  and equals c sum_{q in S} [Re R^q, Im R^q][Re R^q, Im R^q]^T over the half set S.

Two tests model the fp16 slice arithmetic of the tensor-core contractions (E'
and B = M L) and check the exactness and error bounds they rely on; the last
restates the fused finish's 2 x 2 block formulas (E' -> chemist-order ERIs and
the J/K trace terms) and checks them against the direct map and the oracle's
traces.
"""
import numpy as np
import pytest

import oracle as O
from paper_2601_16379_gb300 import workloads as W


def _cell(kmesh):
    shells = [W.Shell(0, 0, (0.6,), (1.0,)), W.Shell(1, 0, (0.9,), (1.0,)), W.Shell(0, 1, (1.2,), (1.0,))]
    return W.custom_cell(5.0, [[0, 0, 0], [0.37, 0.52, 0.21]], shells, kmesh, 10)


def _half_set(kmesh):
    """The q of the paired sum and their weights: m0 in [0, n0/2], and m1 in
    [0, n1/2] when m0 is its own negative; weight 1/2 when m0 and m1 both are."""
    n0, n1, n2 = kmesh
    out = []
    for q in range(n0 * n1 * n2):
        m0, m1 = q // (n1 * n2), (q // n2) % n1
        self0 = m0 == 0 or 2 * m0 == n0
        self1 = m1 == 0 or 2 * m1 == n1
        if 2 * m0 <= n0 and (not self0 or 2 * m1 <= n1):
            out.append((q, 0.5 if (self0 and self1) else 1.0))
    return out


def _rows(nf):
    """Row transform to the time-reversal basis (unnormalised) and its inverse map."""
    n2 = nf * nf
    pairs = [(p, q) for p in range(nf) for q in range(p + 1, nf)]
    P = len(pairs)
    T = np.zeros((n2, n2), np.complex128)
    Cm = np.zeros((n2, n2), np.complex128)
    for o, (p, q) in enumerate(pairs):
        a, s = p * nf + q, q * nf + p
        T[2 * o, a], T[2 * o, s] = 1.0, 1.0            # u = B_(pq) + B_(qp)
        T[2 * o + 1, a], T[2 * o + 1, s] = -1j, 1j      # v = -i (B_(pq) - B_(qp))
        Cm[a, 2 * o], Cm[a, 2 * o + 1] = 0.5, 0.5j
        Cm[s, 2 * o], Cm[s, 2 * o + 1] = 0.5, -0.5j
    for p in range(nf):
        T[2 * P + p, p * nf + p] = 1.0
        Cm[p * nf + p, 2 * P + p] = 1.0
    return T, Cm


@pytest.mark.parametrize("kmesh", [(3, 3, 3), (4, 2, 3)])
def test_real_symmetric_form_of_E(kmesh):
    cell = _cell(kmesh)
    r = O.run_isdf(cell, 12, 7, solve_tol=1e-14)
    nk, nf = cell.nkpts, 4
    frag = W.make_fragment(cell, 11, 2, nf)
    M = O.pair_tensor(O.fragment_T(r["X"], frag.C), cell.kmesh)
    V = r["V"]
    E = O.fragment_E(M, V, nk)
    T, Cm = _rows(nf)
    # any factor of each V^q will do: the identity is one of M V M^H
    Ep = np.zeros((nf * nf, nf * nf))
    for q, w in _half_set(kmesh):
        lam, U = np.linalg.eigh(V[q])
        L = U * np.sqrt(np.clip(lam, 0.0, None))[None, :]
        R = T @ (M[q] @ L)
        Rr = np.hstack([R.real, R.imag])
        Ep += w * Rr @ Rr.T
    Ep *= 2.0 / nk
    scale = np.abs(E).max()
    # E in the time-reversal basis is real and equals the real half-set product
    Et = T @ E @ T.conj().T
    assert np.abs(Et.imag).max() < 1e-10 * scale
    assert np.abs(Et.real - Ep).max() < 1e-10 * scale
    # the finish map E = Cm E' Cm^H recovers E
    assert np.abs(Cm @ Ep @ Cm.conj().T - E).max() < 1e-10 * scale


def test_structural_zeros_of_the_coulomb_factor():
    """L^q = W^T L_xi with W = L_S^{-1} scattered to the pivot columns: its rows
    outside the pivots of Pi^q and its columns beyond the rank of V_xi vanish, and
    M L over the gathered pivot columns equals the full product."""
    cell = _cell((3, 3, 3))
    r = O.run_isdf(cell, 20, 7, solve_tol=1e-6)
    nk = cell.nkpts
    frag = W.make_fragment(cell, 11, 2, 3)
    M = O.pair_tensor(O.fragment_T(r["X"], frag.C), cell.kmesh)
    seen_truncated = False
    for q in range(nk):
        L, perm, rank = O.pchol(r["Pi"][q], 1e-6)
        n = r["Pi"].shape[1]
        seen_truncated |= rank < n
        Wm = np.zeros((n, n), np.complex128)
        LS = L[perm[:rank], :rank]
        Wm[:rank, perm[:rank]] = np.linalg.inv(LS)
        # xi = W eta has zero rows beyond the rank; zeta = W^H xi is the basic solution of the fit
        xi = Wm @ r["eta"][q]
        assert np.abs(xi[rank:]).max() == 0.0
        zeta = Wm.conj().T @ xi
        assert np.abs(zeta - r["zeta"][q]).max() < 1e-8 * np.abs(r["zeta"][q]).max()
        # V_xi = L_xi L_xi^H has rank <= r_q, so L^q = W^T L_xi lives in the pivot rows
        Vx = O.coulomb_metric(cell, xi[None], [q])[0]
        lam, U = np.linalg.eigh(Vx)
        keep = lam > 1e-12 * lam.max()
        Lxi = U[:, keep] * np.sqrt(lam[keep])[None, :]
        Lq = Wm.T @ Lxi
        others = np.setdiff1d(np.arange(n), perm[:rank])
        if others.size:
            assert np.abs(Lq[others]).max() == 0.0
        assert Lxi.shape[1] <= rank
        full = M[q] @ Lq
        gathered = M[q][:, perm[:rank]] @ Lq[perm[:rank]]
        assert np.abs(full - gathered).max() <= 1e-13 * np.abs(full).max()
        # and it reproduces V^q
        assert np.abs(Lq @ Lq.conj().T - r["V"][q]).max() < 1e-8 * np.abs(r["V"][q]).max()
    assert seen_truncated


# ------------------------------------------------------------ slice arithmetic
# The tensor-core contractions of the mixed path write each scaled value x
# (|x| < 128 after the per-row power-of-two scaling) as fp16 slices whose
# products the tcgen05 MMA accumulates in FP32.  These tests model that
# arithmetic in numpy (fp16 rounding of the slices, exact FP64 products) and
# check the facts the kernels rely on.

def _scaled_rows(rng, n, k):
    """Rows of mixed magnitude, each scaled by a power of two so that its largest
    entry lies in [64, 128), as the slicing kernels do; also returns the scales."""
    R = rng.standard_normal((n, k)) * np.exp(rng.uniform(-6.0, 6.0, size=(n, 1)))
    R[:, ::7] *= 1e-3                                    # small entries inside a row
    e = 6 - np.floor(np.log2(np.abs(R).max(axis=1)))
    return (R * 2.0 ** e[:, None]).astype(np.float32).astype(np.float64), 2.0 ** e


def _f16(x):
    return x.astype(np.float16).astype(np.float64)


def test_e_prime_two_slice_form():
    """E' = R R^T from s1 = rint(x) and s2 = fp16(x - s1): the g0 products are
    integers whose partial sums over a 1024-step chunk stay within 2^24 (so their
    FP32 accumulation is exact), the diagonal correction sum x^2 - (s1 + s2)^2
    makes E'_aa exact, and off the diagonal the four products are within 2^-18 of
    |R_a||R_b|."""
    rng = np.random.default_rng(5)
    X, _ = _scaled_rows(rng, 24, 2048)
    assert np.abs(X).max() < 128.0 and np.all(np.abs(X).max(axis=1) >= 64.0)
    s1 = np.rint(X)
    s2 = _f16(X - s1)
    assert np.abs(s1).max() <= 128 and np.abs(s2).max() <= 0.5
    g0 = s1 @ s1.T
    chunk = 1024
    worst = max(np.abs(s1[:, c:c + chunk]).sum(axis=1).max() for c in range(0, X.shape[1], chunk))
    assert worst * 128.0 <= 2.0 ** 24                    # any partial sum of a chunk is an exact FP32 integer
    Ep = g0 + s1 @ s2.T + s2 @ s1.T + s2 @ s2.T
    corr = (X ** 2).sum(axis=1) - ((s1 + s2) ** 2).sum(axis=1)
    Ep[np.diag_indices_from(Ep)] += corr
    E = X @ X.T
    nrm = np.sqrt(np.outer((X ** 2).sum(1), (X ** 2).sum(1)))
    assert np.allclose(np.diag(Ep), np.diag(E), rtol=1e-13, atol=0)   # FP64 summation order only
    assert np.abs(Ep - E).max() / nrm.max() < 2.0 ** -18
    # the remainder's fp16 rounding: unit roundoff 2^-11 of |s2| (2^-25 below fp16's
    # normal range), i.e. ~19 significant bits per value with |x| in [64, 128)
    assert np.all(np.abs(X - s1 - s2) <= 2.0 ** -11 * np.abs(s2) + 2.0 ** -25)


def test_b_three_slice_form():
    """B = M L from an integer and two fp16 remainders per operand (six products,
    i + j <= 2): g0 = S1 T1 stays an exact FP32 integer sum for 2 r_q <= 640, and
    the result is within 2^-26 of |M_a||L_J| (B carries the cancellation of the
    ill-conditioned factor, so the bound is on the operands, not on B)."""
    rng = np.random.default_rng(6)
    A, sa = _scaled_rows(rng, 16, 640)
    Bt, sb = _scaled_rows(rng, 12, 640)
    def sl(x):
        s1 = np.rint(x)
        s2 = _f16(x - s1)
        s3 = _f16(x - s1 - s2)
        return [s1, s2, s3]
    a, b = sl(A), sl(Bt)
    assert 640 * 128.0 * 128.0 <= 2.0 ** 24
    prod = sum(a[i] @ b[j].T for i in range(3) for j in range(3) if i + j <= 2)
    ref = A @ Bt.T
    nrm = np.sqrt(np.outer((A ** 2).sum(1), (Bt ** 2).sum(1)))
    assert np.abs(prod - ref).max() / nrm.max() < 2.0 ** -26


def _block_formulas(Ep, gamma, nf):
    """The E' -> ERI map and the trace terms of the fused finish, block by block:
    orbit o (pair p < q: rows u = 2 o, v = 2 o + 1; diagonal p: row 2 P + p), the
    block of two orbits U = E'(u1, u2), X = E'(u1, v2), Y = E'(v1, u2), Z = E'(v1, v2),
    and the real-part trace formulas for a Hermitian gamma."""
    pairs = [(p, q) for p in range(nf) for q in range(p + 1, nf)]
    P = len(pairs)
    orbs = pairs + [(p, p) for p in range(nf)]
    row = lambda o: 2 * o if o < P else 2 * P + (o - P)
    eri = np.zeros((nf,) * 4, complex)
    aj = ak = 0.0
    g = gamma
    for o1, (p, q) in enumerate(orbs):
        for o2, (x, y) in enumerate(orbs):
            u1, u2 = row(o1), row(o2)
            pr, pc = p != q, x != y
            U = Ep[u1, u2]
            X = Ep[u1, u2 + 1] if pc else 0.0
            Y = Ep[u1 + 1, u2] if pr else 0.0
            Z = Ep[u1 + 1, u2 + 1] if pr and pc else 0.0
            if pr and pc:
                r1, i1, r2, i2 = (U + Z) / 4, (Y - X) / 4, (U - Z) / 4, (X + Y) / 4
                eri[p, q, y, x], eri[p, q, x, y] = r1 + 1j * i1, r2 + 1j * i2
                eri[q, p, y, x], eri[q, p, x, y] = r2 - 1j * i2, r1 - 1j * i1
                A, B = g[p, q], g[y, x]
                aj += U * A.real * B.real - Z * A.imag * B.imag + X * A.real * B.imag - Y * A.imag * B.real
                w1, w2 = g[p, x] * g[y, q], g[p, y] * g[x, q]
                ak += 2 * (w1.real * r1 - w1.imag * i1 + w2.real * r2 - w2.imag * i2)
            elif pr:
                r, im = U / 2, Y / 2
                eri[p, q, x, x], eri[q, p, x, x] = r + 1j * im, r - 1j * im
                A = g[p, q]
                aj += g[x, x].real * (A.real * U - A.imag * Y)
                w = g[p, x] * g[x, q]
                ak += 2 * (w.real * r - w.imag * im)
            elif pc:
                r, im = U / 2, -X / 2
                eri[p, p, y, x], eri[p, p, x, y] = r + 1j * im, r - 1j * im
                B = g[y, x]
                aj += g[p, p].real * (B.real * U + B.imag * X)
                w = g[p, x] * g[y, p]
                ak += 2 * (w.real * r - w.imag * im)
            else:
                eri[p, p, x, x] = U
                w = g[p, x]
                aj += g[p, p].real * g[x, x].real * U
                ak += abs(w) ** 2 * U
    return eri, 0.5 * aj, -0.25 * ak


def test_finish_block_formulas_equal_direct_map():
    """The finish never forms E: it maps each 2 x 2 block of the real E' straight to
    chemist-order ERIs and trace terms.  On a random real symmetric E' and a random
    Hermitian gamma those formulas equal E = T^-1 E' T^-H with the time-reversal
    basis rows u = e_(pq) + e_(qp), v = -i (e_(pq) - e_(qp)), e_(pp), the chemist
    order (pq|rs) = E_(pq),(sr), and the oracle's direct traces."""
    rng = np.random.default_rng(8)
    nf = 5
    n2 = nf * nf
    pairs = [(p, q) for p in range(nf) for q in range(p + 1, nf)]
    T = np.zeros((n2, n2), complex)
    for o, (p, q) in enumerate(pairs):
        T[2 * o, p * nf + q] = T[2 * o, q * nf + p] = 1.0
        T[2 * o + 1, p * nf + q], T[2 * o + 1, q * nf + p] = -1j, 1j
    for p in range(nf):
        T[2 * len(pairs) + p, p * nf + p] = 1.0
    A = rng.standard_normal((n2, n2))
    Ep = A @ A.T
    Ti = np.linalg.inv(T)
    E = Ti @ Ep @ Ti.conj().T
    s = np.array([q * nf + p for p in range(nf) for q in range(nf)])   # (pq) -> (qp)
    assert np.allclose(E[np.ix_(s, s)], E.conj())                       # the time-reversal symmetry
    ref = O.eri_from_E(E, nf)
    G = rng.standard_normal((nf, nf)) + 1j * rng.standard_normal((nf, nf))
    gamma = G @ G.conj().T
    rj, rk = O.traces(ref, gamma)
    eri, ej, ek = _block_formulas(Ep, gamma, nf)
    assert np.abs(eri - ref).max() < 1e-12 * np.abs(ref).max()
    assert abs(ej - rj) < 1e-11 * abs(rj) and abs(ek - rk) < 1e-11 * abs(rk)
