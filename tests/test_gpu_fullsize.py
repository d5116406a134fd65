"""Full-size checks at the c4 workload (Nk = 216, 24^3 grid, N_P = 300) and,
at the end of the file, at c3 (52 AOs, Nk = 64, 32^3 grid, N_P = 500). c4 runs in the
launch configuration that bench.py times (mixed precision, tensor-core
contraction, all steps).

The FP64 oracle cannot run c4's fit in test time, so these checks use
(1) the oracle on outputs it can compute one by one: Bloch GTOs at the
interpolation points for sampled k-points; (2) the GPU FP64 path, itself
checked against the oracle on c1, c2 and the anisotropic cell, for fragments
of the smallest, median and a mid-large size: mixed and FP64 ERIs and traces
must agree to the mixed tolerance; (3) properties that hold at any size:
Hermitian E with non-negative diagonal and PSD 2x2 minors, (pq|rs) = (rs|pq)
= conj((qp|sr)) on sampled entries, E_J > 0 > E_K.
"""
import numpy as np
import pytest

import oracle as O
from paper_2601_16379_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-6
TAU = 1e-7


@pytest.fixture(scope="module")
def c4_runs(cuda, lib_built):
    from paper_2601_16379_gb300 import binding as B
    torch = cuda
    wl = W.workload("c4", with_fragments=False)
    sizes = wl.frag_sizes
    order = np.argsort(sizes)
    pick = [int(order[0]), int(order[len(order) // 2]), int(order[int(0.7 * len(order))])]
    frags = W.make_fragments(wl, pick)
    out = {}
    ips = None
    for prec in (B.ISDF_MIXED, B.ISDF_FP64):
        g = B.Isdf(wl.cell, prec)
        got = g.build_points(wl.n_p, wl.seed)
        if ips is None:
            ips = got
        else:
            assert np.array_equal(ips, got)
        s = g.sizes()
        X = torch.empty((s["nk"], s["np"], s["nao"]), dtype=torch.complex128, device="cuda")
        g.get(0, X)
        g.fit_zeta(TAU)
        V = torch.empty((s["nk"], s["np"], s["np"]), dtype=torch.complex128, device="cuda")
        g.coulomb_metric(V)
        dt = torch.complex64 if prec == B.ISDF_MIXED else torch.complex128
        Cs = [torch.from_numpy(f.C).cuda() for f in frags]
        gs = [torch.from_numpy(f.gamma).cuda() for f in frags]
        eris = [torch.empty((f.norb,) * 4, dtype=dt, device="cuda") for f in frags]
        ej, ek = g.fragment_eri(Cs, gs, eris)
        torch.cuda.synchronize()
        out[prec] = dict(X=X.cpu().numpy(), V=V.cpu().numpy(),
                         eri=[e.cpu().numpy().astype(np.complex128) for e in eris], ej=ej, ek=ek)
        del V
        g.close()
    return wl, frags, ips, out


def test_interp_vectors_against_oracle(c4_runs):
    """X^k_{I mu} = phi^k_mu(r_I) (Eq. 1) for sampled k, all points: the oracle
    evaluates the lattice sums at the selected grid points."""
    from paper_2601_16379_gb300 import binding as B
    wl, frags, ips, out = c4_runs
    pts = O.grid_points(wl.cell)[ips]
    ks = [0, 7, 101, 215]
    phi = O.bloch_ao(wl.cell, kidx=ks, pts=pts)          # (len(ks), N_AO, N_P)
    Xo = phi.transpose(0, 2, 1)
    Xg = out[B.ISDF_MIXED]["X"][ks]
    assert np.abs(Xg - Xo).max() <= 1e-13 * np.abs(Xo).max()


def test_smallest_fragment_against_oracle(c4_runs):
    """The whole smallest c4 fragment (ERIs, E_J, E_K) against the oracle's direct
    k-sums (Eqs. 19-20) given the FP64 path's X^k and V^q, in both precisions, and
    its E_J against the oracle's cheap-J identity (a^Q = sum gamma_pq M^Q_(pq),
    E_J = sum_Q a^Q V^Q a^Q^H / 2Nk), which needs no ERIs."""
    from paper_2601_16379_gb300 import binding as B
    wl, frags, ips, out = c4_runs
    d = out[B.ISDF_FP64]
    f = frags[0]
    ref = O.fragment_eri(d["X"], d["V"], f.C, wl.cell.kmesh)
    rj, rk = O.traces(ref, f.gamma)
    for prec, tol in ((B.ISDF_FP64, 1e-8), (B.ISDF_MIXED, MIXED_TOL)):
        assert np.abs(out[prec]["eri"][0] - ref).max() < tol
        assert abs(out[prec]["ej"][0] - rj) < tol and abs(out[prec]["ek"][0] - rk) < tol
    M = O.pair_tensor(O.fragment_T(d["X"], f.C), wl.cell.kmesh)
    cj = O.cheap_J(M, d["V"], f.gamma, wl.cell.nkpts)
    assert abs(d["ej"][0] - cj) < 1e-8 and abs(out[B.ISDF_MIXED]["ej"][0] - cj) < MIXED_TOL


def test_mixed_matches_fp64_path(c4_runs):
    from paper_2601_16379_gb300 import binding as B
    wl, frags, ips, out = c4_runs
    m, d = out[B.ISDF_MIXED], out[B.ISDF_FP64]
    for i in range(len(frags)):
        assert np.abs(m["eri"][i] - d["eri"][i]).max() < MIXED_TOL
        assert abs(m["ej"][i] - d["ej"][i]) < MIXED_TOL
        assert abs(m["ek"][i] - d["ek"][i]) < MIXED_TOL


def test_properties_at_full_size(c4_runs):
    from paper_2601_16379_gb300 import binding as B
    wl, frags, ips, out = c4_runs
    rng = np.random.default_rng(3)
    for prec in (B.ISDF_MIXED, B.ISDF_FP64):
        tol = 1e-6 if prec == B.ISDF_MIXED else 1e-10
        for i, f in enumerate(frags):
            e = out[prec]["eri"][i]
            n = f.norb
            s = np.abs(e).max()
            idx = rng.integers(0, n, size=(2000, 4))
            p, q, r, t = idx.T
            assert np.abs(e[p, q, r, t] - e[r, t, p, q]).max() < tol * s
            assert np.abs(e[p, q, r, t] - np.conj(e[q, p, t, r])).max() < tol * s
            # H_(ab),(cd) = (ba|cd) is Hermitian PSD: diagonal >= 0 and |H_xy|^2 <= H_xx H_yy
            diag = np.array([[e[b, a, a, b] for b in range(n)] for a in range(n)]).real  # H_(ab),(ab)
            assert diag.min() > -tol * s
            a, b, c, dd = idx.T
            hxy = e[b, a, c, dd]
            hxx = np.array([e[bb, aa, aa, bb] for aa, bb in zip(a, b)]).real
            hyy = np.array([e[dd_, cc, cc, dd_] for cc, dd_ in zip(c, dd)]).real
            assert np.all(np.abs(hxy) ** 2 <= hxx * hyy * (1 + 1e-6) + tol * s * s)
            assert out[prec]["ej"][i] > 0 > out[prec]["ek"][i]


@pytest.fixture(scope="module")
def c3_runs(cuda, lib_built):
    """c3 at its own size (52 AOs, 4x4x4 mesh, 32^3 grid, N_P = 500, 3 fragments of 60):
    N_P = 500 puts B = M L on the compensated SIMT GEMM in the mixed path."""
    from paper_2601_16379_gb300 import binding as B
    torch = cuda
    wl = W.workload("c3")
    out = {}
    for prec in (B.ISDF_MIXED, B.ISDF_FP64):
        g = B.Isdf(wl.cell, prec)
        g.build_points(wl.n_p, wl.seed)
        g.fit_zeta(TAU)
        g.coulomb_metric()
        dt = torch.complex64 if prec == B.ISDF_MIXED else torch.complex128
        Cs = [torch.from_numpy(f.C).cuda() for f in wl.fragments]
        gs = [torch.from_numpy(f.gamma).cuda() for f in wl.fragments]
        eris = [torch.empty((f.norb,) * 4, dtype=dt, device="cuda") for f in wl.fragments]
        ej, ek = g.fragment_eri(Cs, gs, eris)
        torch.cuda.synchronize()
        out[prec] = dict(eri=[e.cpu().numpy().astype(np.complex128) for e in eris], ej=ej, ek=ek)
        g.close()
    return wl, out


def test_c3_mixed_matches_fp64_and_symmetries(c3_runs):
    from paper_2601_16379_gb300 import binding as B
    wl, out = c3_runs
    m, d = out[B.ISDF_MIXED], out[B.ISDF_FP64]
    for i, f in enumerate(wl.fragments):
        assert np.abs(m["eri"][i] - d["eri"][i]).max() < MIXED_TOL
        assert abs(m["ej"][i] - d["ej"][i]) < MIXED_TOL and abs(m["ek"][i] - d["ek"][i]) < MIXED_TOL
        e = d["eri"][i]
        s = np.abs(e).max()
        assert np.abs(e - e.transpose(2, 3, 0, 1)).max() < 1e-10 * s       # (pq|rs) = (rs|pq)
        assert np.abs(e - e.transpose(1, 0, 3, 2).conj()).max() < 1e-10 * s  # = conj((qp|sr))
        assert d["ej"][i] > 0 > d["ek"][i]
