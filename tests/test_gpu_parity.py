"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: the FP64 path and the FP64-class tensor-core path (FP64_TC) must
match the oracle to 1e-8 Ha in every ERI and in E_J / E_K; the mixed path to
1e-6 Ha.  Integer work (interpolation points,
ranks) must match exactly.  Intermediate arrays of the fit match to ~1e-13
relative (same FP64 arithmetic in a different order).

The solve tolerance tau of the Pi^q factorisation is part of the problem: the
basic least-squares solution changes discontinuously when a pivot crosses tau,
so parity cases use tau values where rounding-level differences cannot move a
pivot across it (tie windows handle exact symmetry ties).
"""
import numpy as np
import pytest

import oracle as O
from paper_2601_16379_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-8
MIXED_TOL = 1e-6


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_eri(torch, g, frags, prec):
    dt = torch.complex64 if prec == 1 else torch.complex128
    Cs = [_dev(torch, f.C) for f in frags]
    gs = [_dev(torch, f.gamma) for f in frags]
    outs = [torch.empty((f.norb,) * 4, dtype=dt, device="cuda") for f in frags]
    ej, ek = g.fragment_eri(Cs, gs, outs)
    torch.cuda.synchronize()
    return [o.cpu().numpy().astype(np.complex128) for o in outs], ej, ek


class OracleRun:
    def __init__(self, cell, n_p, seed, ips=None):
        self.cell = cell
        self.phi = O.bloch_ao(cell)
        if ips is None:
            ips, nf = O.select_ips(self.phi, n_p, seed)
            assert nf == n_p
        self.ips = ips
        self.X = O.interp_vectors(self.phi, ips)
        self.Pi = O.metric_pi(self.X, cell.kmesh)
        self.eta = O.rhs_eta(self.X, self.phi, cell.kmesh)
        self._fits = {}

    def fit(self, tol):
        if tol not in self._fits:
            zeta, ranks = O.fit_zeta(self.Pi, self.eta, tol)
            V = O.coulomb_metric(self.cell, zeta, range(self.cell.nkpts))
            self._fits[tol] = (zeta, ranks, V)
        return self._fits[tol]

    def eri(self, tol, f):
        _, _, V = self.fit(tol)
        e = O.fragment_eri(self.X, V, f.C, self.cell.kmesh)
        return e, O.traces(e, f.gamma)


def aniso_cell():
    sh = [W.Shell(0, 0, (0.6,), (1.0,)), W.Shell(1, 1, (0.9,), (1.0,)), W.Shell(1, 2, (1.1,), (0.7,))]
    return W.custom_cell(5.0, [[0, 0, 0], [0.37, 0.52, 0.21]], sh, (2, 1, 3), (12, 10, 14))


@pytest.fixture(scope="module")
def c1():
    wl = W.workload("c1")
    return wl, OracleRun(wl.cell, wl.n_p, wl.seed)


@pytest.fixture(scope="module")
def aniso():
    cell = aniso_cell()
    return cell, OracleRun(cell, 40, 99)


@pytest.fixture(scope="module")
def c2():
    wl = W.workload("c2")
    return wl, OracleRun(wl.cell, wl.n_p, wl.seed)


# ------------------------------------------------------------------ points
def test_points_bit_exact_c1(cuda, lib_built, c1):
    from paper_2601_16379_gb300 import binding as B
    wl, o = c1
    g = B.Isdf(wl.cell, B.ISDF_FP64)
    assert np.array_equal(g.build_points(wl.n_p, wl.seed), o.ips)


def test_points_bit_exact_aniso(cuda, lib_built, aniso):
    from paper_2601_16379_gb300 import binding as B
    cell, o = aniso
    g = B.Isdf(cell, B.ISDF_FP64)
    assert np.array_equal(g.build_points(40, 99), o.ips)


def test_points_c2(cuda, lib_built, c2):
    from paper_2601_16379_gb300 import binding as B
    wl, o = c2
    g = B.Isdf(wl.cell, B.ISDF_FP64)
    assert np.array_equal(g.build_points(wl.n_p, wl.seed), o.ips)


# ----------------------------------------------------------- intermediates
def test_fit_intermediates_c1(cuda, lib_built, c1):
    from paper_2601_16379_gb300 import binding as B
    torch = cuda
    wl, o = c1
    g = B.Isdf(wl.cell, B.ISDF_FP64)
    g.set_points(o.ips)
    s = g.sizes()
    nk, npp, nao, ng = s["nk"], s["np"], s["nao"], s["ng"]
    X = g.get(0, torch.empty((nk, npp, nao), dtype=torch.complex128, device="cuda")).cpu().numpy()
    assert np.abs(X - o.X).max() <= 1e-14 * np.abs(o.X).max()
    ranks = g.fit_zeta(1e-7)
    assert np.array_equal(ranks, o.fit(1e-7)[1])
    Pi = g.get(1, torch.empty((nk, npp, npp), dtype=torch.complex128, device="cuda")).cpu().numpy()
    assert np.abs(Pi - o.Pi).max() <= 1e-13 * np.abs(o.Pi).max()
    eta = g.get(2, torch.empty((nk, npp, ng), dtype=torch.complex128, device="cuda")).cpu().numpy()
    assert np.abs(eta - o.eta).max() <= 1e-13 * np.abs(o.eta).max()


def test_zeta_and_V_full_rank(cuda, lib_built, aniso):
    """Where every Pi^q has full rank the solution is unique: zeta and V match."""
    from paper_2601_16379_gb300 import binding as B
    torch = cuda
    cell, o = aniso
    tol = 1e-12
    zeta, ranks, V = o.fit(tol)
    assert ranks.min() == 40
    g = B.Isdf(cell, B.ISDF_FP64)
    g.set_points(o.ips)
    g.fit_zeta(tol)
    nk, ng = cell.nkpts, cell.ngrid
    z = g.get(3, torch.empty((nk, 40, ng), dtype=torch.complex128, device="cuda")).cpu().numpy()
    assert np.abs(z - zeta).max() <= 1e-5 * np.abs(zeta).max()
    Vg = torch.empty((nk, 40, 40), dtype=torch.complex128, device="cuda")
    g.coulomb_metric(Vg)
    Vg = Vg.cpu().numpy()
    assert np.abs(Vg - V).max() <= 1e-5 * np.abs(V).max()


# ------------------------------------------------------------ fragment ERIs
@pytest.mark.parametrize("tol", [1e-7])
def test_fp64_eri_c1(cuda, lib_built, c1, tol):
    from paper_2601_16379_gb300 import binding as B
    wl, o = c1
    frags = list(wl.fragments) + [W.make_fragment(wl.cell, wl.seed, 5, 7), W.make_fragment(wl.cell, wl.seed, 6, 1)]
    g = B.Isdf(wl.cell, B.ISDF_FP64)
    g.build_points(wl.n_p, wl.seed)
    g.fit_zeta(tol)
    g.coulomb_metric()
    eris, ej, ek = gpu_eri(cuda, g, frags, 0)
    for i, f in enumerate(frags):
        ref, (rj, rk) = o.eri(tol, f)
        assert np.abs(eris[i] - ref).max() < FP64_TOL
        assert abs(ej[i] - rj) < FP64_TOL and abs(ek[i] - rk) < FP64_TOL


def test_fp64_eri_aniso(cuda, lib_built, aniso):
    from paper_2601_16379_gb300 import binding as B
    cell, o = aniso
    frags = [W.make_fragment(cell, 5, 0, 5), W.make_fragment(cell, 5, 1, 2)]
    g = B.Isdf(cell, B.ISDF_FP64)
    g.build_points(40, 99)
    g.fit_zeta(1e-12)
    g.coulomb_metric()
    eris, ej, ek = gpu_eri(cuda, g, frags, 0)
    for i, f in enumerate(frags):
        ref, (rj, rk) = o.eri(1e-12, f)
        assert np.abs(eris[i] - ref).max() < FP64_TOL
        assert abs(ej[i] - rj) < FP64_TOL and abs(ek[i] - rk) < FP64_TOL


def test_mixed_eri_c1(cuda, lib_built, c1):
    from paper_2601_16379_gb300 import binding as B
    wl, o = c1
    tol = 1e-7
    frags = list(wl.fragments) + [W.make_fragment(wl.cell, wl.seed, 5, 7)]
    g = B.Isdf(wl.cell, B.ISDF_MIXED)
    g.build_points(wl.n_p, wl.seed)
    g.fit_zeta(tol)
    g.coulomb_metric()
    eris, ej, ek = gpu_eri(cuda, g, frags, 1)
    for i, f in enumerate(frags):
        ref, (rj, rk) = o.eri(tol, f)
        assert np.abs(eris[i] - ref).max() < MIXED_TOL
        assert abs(ej[i] - rj) < MIXED_TOL and abs(ek[i] - rk) < MIXED_TOL


@pytest.mark.parametrize("prec", [0, 1])
def test_time_reversal_pairing_matches_full_sum(cuda, lib_built, c2, prec):
    """The contraction over about half of the q-points completed by the
    (pq) -> (qp) conjugate swap (15 of the 27 q-points on the 3x3x3 mesh) gives
    the ERIs and traces of the sum over all q, and both match the oracle."""
    from paper_2601_16379_gb300 import binding as B
    wl, o = c2
    tol = 1e-7
    res = {}
    for pair in (True, False):
        g = B.Isdf(wl.cell, prec)
        g.set_time_reversal(pair)
        g.build_points(wl.n_p, wl.seed)
        g.fit_zeta(tol)
        g.coulomb_metric()
        res[pair] = gpu_eri(cuda, g, wl.fragments, prec)
        g.close()
    bound = FP64_TOL if prec == 0 else MIXED_TOL
    for i, f in enumerate(wl.fragments):
        ref, (rj, rk) = o.eri(tol, f)
        for pair in (True, False):
            eris, ej, ek = res[pair]
            assert np.abs(eris[i] - ref).max() < bound
            assert abs(ej[i] - rj) < bound and abs(ek[i] - rk) < bound
        assert np.abs(res[True][0][i] - res[False][0][i]).max() < bound
        assert abs(res[True][1][i] - res[False][1][i]) < bound


@pytest.mark.parametrize("qc", [1, 4])
def test_mixed_q_chunks_c2(cuda, lib_built, c2, qc):
    """The mixed contraction taken in q-chunks (qc q-points of B per launch; the
    15 paired q-points of the 3x3x3 mesh give a ragged last chunk for qc = 4)
    accumulates the same E as one launch over all of them, and stays within the
    mixed tolerance of the oracle."""
    from paper_2601_16379_gb300 import binding as B
    wl, o = c2
    tol = 1e-7
    f = wl.fragments[0]
    n2, np_ = f.norb ** 2, wl.n_p
    k2 = -(-2 * np_ // 64) * 64                 # fp16 columns of one q-point, padded to 64
    per_q = 3 * n2 * k2 * 2 + 256                 # three slices of M (B = M L), the larger per-q buffer
    res = {}
    for limit in (None, qc * per_q):
        g = B.Isdf(wl.cell, B.ISDF_MIXED)
        if limit is not None:
            g.set_workspace_limit(1 if qc == 1 else limit)
        g.build_points(wl.n_p, wl.seed)
        g.fit_zeta(tol)
        g.coulomb_metric()
        res[limit] = gpu_eri(cuda, g, [f], 1)
        g.close()
    one, chunked = res[None], res[qc * per_q]
    # the ERIs are returned in complex64: allow two fp32 ulps at the largest entry.
    # The traces are reduced in FP64 from E'; the exact g0 products are independent of
    # the chunking, but the low-order group g1 (products with the fp16 remainders,
    # 2^-7 of the total) accumulates in FP32, whose rounding depends on where the
    # chunks start: ~2^-24 per accumulation, 1e-8 of E_J bounds it
    scale = np.abs(one[0][0]).max()
    assert np.abs(chunked[0][0] - one[0][0]).max() <= 2.4e-7 * scale
    tr = 1e-8 * abs(one[1][0])
    assert abs(chunked[1][0] - one[1][0]) < tr and abs(chunked[2][0] - one[2][0]) < tr
    ref, (rj, rk) = o.eri(tol, f)
    assert np.abs(chunked[0][0] - ref).max() < MIXED_TOL
    assert abs(chunked[1][0] - rj) < MIXED_TOL and abs(chunked[2][0] - rk) < MIXED_TOL


def test_mixed_large_np_matches_fp64(cuda, lib_built):
    """N_P = 520 puts B = M L (K' = 2 N_P > 1024) on the compensated SIMT GEMM
    instead of the exact-slice tensor kernel; the mixed ERIs and traces still
    match the FP64 path (itself pinned to the oracle) within the mixed bound."""
    from paper_2601_16379_gb300 import binding as B
    wl = W.workload("c3", kmesh=2, mesh=24, n_p=520, frag_sizes=[6, 9])
    res = {}
    for prec in (B.ISDF_FP64, B.ISDF_MIXED):
        g = B.Isdf(wl.cell, prec)
        g.build_points(wl.n_p, wl.seed)
        g.fit_zeta(1e-7)
        g.coulomb_metric()
        res[prec] = gpu_eri(cuda, g, wl.fragments, prec)
        g.close()
    d, m = res[B.ISDF_FP64], res[B.ISDF_MIXED]
    for i in range(len(wl.fragments)):
        assert np.abs(m[0][i] - d[0][i]).max() < MIXED_TOL
        assert abs(m[1][i] - d[1][i]) < MIXED_TOL and abs(m[2][i] - d[2][i]) < MIXED_TOL


@pytest.mark.parametrize("prec", [0, 1])
def test_eri_out_in_pinned_host_memory(cuda, lib_built, c1, prec):
    """eri_out may be page-locked host memory: the result equals the device one."""
    from paper_2601_16379_gb300 import binding as B
    torch = cuda
    wl, o = c1
    f = W.make_fragment(wl.cell, wl.seed, 5, 7)
    g = B.Isdf(wl.cell, prec)
    g.build_points(wl.n_p, wl.seed)
    g.fit_zeta(1e-7)
    g.coulomb_metric()
    dt = torch.complex64 if prec == 1 else torch.complex128
    C, gm = _dev(torch, f.C), _dev(torch, f.gamma)
    dev = torch.empty((f.norb,) * 4, dtype=dt, device="cuda")
    host = torch.empty((f.norb,) * 4, dtype=dt).pin_memory()
    ej1, ek1 = g.fragment_eri([C], [gm], [dev])
    ej2, ek2 = g.fragment_eri([C], [gm], [host])
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), host.numpy())
    assert ej1[0] == ej2[0] and ek1[0] == ek2[0]
    g.close()


@pytest.mark.parametrize("case", ["c1", "aniso"])
def test_ao_quartet_eri_matches_oracle(cuda, lib_built, c1, aniso, case):
    """AO-level integrals for k-quartets (Eq. 9) against the oracle, including
    quartets whose Q lies in the conjugated half of the mesh; a quartet that does
    not conserve crystal momentum is refused."""
    from paper_2601_16379_gb300 import binding as B
    torch = cuda
    if case == "c1":
        wl, o = c1
        cell = wl.cell
    else:
        cell, o = aniso
    tol = 1e-7
    _, _, V = o.fit(tol)
    kp, km = O.k_plus_table(cell.kmesh), O.k_minus_table(cell.kmesh)
    nk = cell.nkpts
    quartets = [(0, 0, 0, 0), (1, 0, 0, kp[0, 1]), (nk - 1, 2 % nk, 3 % nk, kp[3 % nk, km[nk - 1, 2 % nk]]),
                (2 % nk, nk - 1, 4 % nk, kp[4 % nk, km[2 % nk, nk - 1]])]
    ref = O.ao_eri(o.X, V, quartets, cell.kmesh)
    g = B.Isdf(cell, B.ISDF_FP64)
    g.set_points(o.ips)
    g.fit_zeta(tol)
    g.coulomb_metric()
    nao = cell.nao
    out = torch.empty((len(quartets), nao, nao, nao, nao), dtype=torch.complex128, device="cuda")
    g.ao_eri(quartets, out)
    got = out.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()
    bad = [(1, 0, 0, 0)] if nk > 1 else None
    if bad:
        with pytest.raises(B.IsdfError) as e:
            g.ao_eri(bad, torch.empty((1, nao, nao, nao, nao), dtype=torch.complex128, device="cuda"))
        assert e.value.code == -1
    g.close()


@pytest.mark.parametrize("case", ["c1", "aniso"])
def test_sos_polarizability_matches_oracle(cuda, lib_built, c1, aniso, case):
    """k-SOS-MP2 polarisability chi^Q(tau) for every Q and the opposite-spin trace
    S(tau) (Eqs. 11-15) against the oracle's direct k-sums, with seeded stand-ins
    for the k-HF orbitals and energies."""
    from paper_2601_16379_gb300 import binding as B
    torch = cuda
    if case == "c1":
        wl, o = c1
        cell = wl.cell
    else:
        cell, o = aniso
    tol = 1e-7
    _, _, V = o.fit(tol)
    C = W.mo_coefficients(cell, 17)
    n_occ = 3
    eps = W.orbital_energies(cell, 17, n_occ)
    g = B.Isdf(cell, B.ISDF_FP64)
    g.set_points(o.ips)
    g.fit_zeta(tol)
    g.coulomb_metric()
    nk, npp = cell.nkpts, len(o.ips)
    Cd = _dev(torch, C)
    for tau in (0.0, 0.6):
        Go, Gv = O.green_ip(o.X, C, eps, n_occ, tau)
        chi_ref = O.polarizability(Go, Gv, cell.kmesh)
        s_ref = O.sos_trace(chi_ref, V, cell.kmesh)
        chi = torch.empty((nk, npp, npp), dtype=torch.complex128, device="cuda")
        s = g.sos_polarizability(Cd, eps, n_occ, tau, chi)
        got = chi.cpu().numpy()
        assert np.abs(got - chi_ref).max() <= 1e-12 * np.abs(chi_ref).max()
        assert abs(s - s_ref) <= 1e-8 * abs(s_ref)
    g.close()


# FP64_TC is tested at tau = 1e-7 (its contraction is exact to ~2^-35 of |M_a||L_J| in
# B = M L, and |L| grows like tau^-1/2: at tau = 1e-12 its E_J is off by ~2e-7 Ha on c2)
@pytest.mark.parametrize("prec,tol", [(0, 1e-7), (0, 1e-12), (1, 1e-7), (2, 1e-7)])
def test_eri_c2(cuda, lib_built, c2, prec, tol):
    from paper_2601_16379_gb300 import binding as B
    wl, o = c2
    g = B.Isdf(wl.cell, prec)
    g.build_points(wl.n_p, wl.seed)
    g.fit_zeta(tol)
    g.coulomb_metric()
    eris, ej, ek = gpu_eri(cuda, g, wl.fragments, prec)
    bound = MIXED_TOL if prec == 1 else FP64_TOL
    for i, f in enumerate(wl.fragments):
        ref, (rj, rk) = o.eri(tol, f)
        assert np.abs(eris[i] - ref).max() < bound
        assert abs(ej[i] - rj) < bound and abs(ek[i] - rk) < bound


# -------------------------------------------------------------- edge cases
def test_gamma_only_and_general_lattice(cuda, lib_built):
    """Nk = 1 (textbook Gamma-point ISDF) on a non-orthorhombic (fcc primitive) cell,
    which takes the direct 3-D lattice-sum kernel."""
    from paper_2601_16379_gb300 import binding as B
    a = 6.0
    lat = 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    cell = W.Cell(lat, np.array([[0.0, 0.0, 0.0], [0.25 * a, 0.25 * a, 0.25 * a]]),
                  [W.Shell(0, 0, (0.7,), (1.0,)), W.Shell(1, 1, (1.0,), (1.0,))], (1, 1, 1), (10, 10, 10))
    for km, n_p in (((1, 1, 1), 8), ((2, 2, 1), 16)):   # 4 real AOs at Gamma: pair rank 10
        cell.kmesh = km
        o = OracleRun(cell, n_p, 4)
        g = B.Isdf(cell, B.ISDF_FP64)
        assert np.array_equal(g.build_points(n_p, 4), o.ips)
        g.fit_zeta(1e-10)
        g.coulomb_metric()
        f = W.make_fragment(cell, 9, 0, 3)
        eris, ej, ek = gpu_eri(cuda, g, [f], 0)
        ref, (rj, rk) = o.eri(1e-10, f)
        assert np.abs(eris[0] - ref).max() < FP64_TOL
        assert abs(ej[0] - rj) < FP64_TOL and abs(ek[0] - rk) < FP64_TOL


def test_repeat_is_bitwise_deterministic(cuda, lib_built, c1):
    from paper_2601_16379_gb300 import binding as B
    wl, o = c1
    outs = []
    for _ in range(2):
        g = B.Isdf(wl.cell, B.ISDF_FP64)
        g.build_points(wl.n_p, wl.seed)
        g.fit_zeta(1e-7)
        g.coulomb_metric()
        outs.append(gpu_eri(cuda, g, wl.fragments, 0))
    assert np.array_equal(outs[0][0][0], outs[1][0][0])
    assert outs[0][1][0] == outs[1][1][0] and outs[0][2][0] == outs[1][2][0]


def test_errors_and_state(cuda, lib_built, c1):
    from paper_2601_16379_gb300 import binding as B
    wl, o = c1
    g = B.Isdf(wl.cell, B.ISDF_FP64)
    with pytest.raises(B.IsdfError) as e:
        g.fit_zeta(1e-7)
    assert e.value.code == -6
    with pytest.raises(B.IsdfError) as e:
        g.coulomb_metric()
    assert e.value.code == -6
    with pytest.raises(B.IsdfError) as e:
        g.build_points(wl.cell.ngrid + 1, 1)
    assert e.value.code == -1
    with pytest.raises(B.IsdfError) as e:
        g.set_points([1, 2, 2])
    assert e.value.code == -1
    with pytest.raises(B.IsdfError) as e:
        g.build_points(4000, wl.seed, chol_tol=1e-2)   # runs out of rank
    assert e.value.code == -4
    g.build_points(wl.n_p, wl.seed)
    g.fit_zeta(1e-7)
    g.coulomb_metric()
    ej, ek = g.fragment_eri([])
    assert len(ej) == 0


# ------------------------------------------------- Coulomb kernel from eta
@pytest.mark.parametrize("case", ["c1", "aniso"])
def test_eta_route_matches_oracle(cuda, lib_built, c1, aniso, case):
    """isdf_coulomb_metric_eta (Eqs. 7-8) gives the fragment ERIs of the zeta
    route (Eq. 6) within the FP64 tolerance at tau = 1e-8 (the eta route
    multiplies rounding by cond(Pi^q), so it is used with a truncation)."""
    from paper_2601_16379_gb300 import binding as B
    tau = 1e-8
    if case == "c1":
        wl, o = c1
        cell, n_p, seed = wl.cell, wl.n_p, wl.seed
        frags = [wl.fragments[0], W.make_fragment(cell, seed, 5, 7)]
    else:
        cell, o = aniso
        n_p, seed = 40, 99
        frags = [W.make_fragment(cell, 5, 0, 5)]
    g = B.Isdf(cell, B.ISDF_FP64)
    g.build_points(n_p, seed)
    g.fit_zeta(tau)
    g.coulomb_metric_eta()
    eris, ej, ek = gpu_eri(cuda, g, frags, 0)
    for i, f in enumerate(frags):
        ref, (rj, rk) = o.eri(tau, f)
        assert np.abs(eris[i] - ref).max() < FP64_TOL
        assert abs(ej[i] - rj) < FP64_TOL and abs(ek[i] - rk) < FP64_TOL


# ------------------------------------------------------ exchange (Eq. 10)
@pytest.mark.parametrize("case,tau", [("c1", 1e-7), ("aniso", 1e-12)])
def test_exchange_matches_oracle(cuda, lib_built, c1, aniso, case, tau):
    from paper_2601_16379_gb300 import binding as B
    torch = cuda
    if case == "c1":
        wl, o = c1
        cell, n_p, seed = wl.cell, wl.n_p, wl.seed
    else:
        cell, o = aniso
        n_p, seed = 40, 99
    rng = np.random.default_rng(11)
    Cs = rng.standard_normal((cell.nkpts, cell.nao, 3)) + 1j * rng.standard_normal((cell.nkpts, cell.nao, 3))
    P = np.einsum("kmi,kni->kmn", Cs, Cs.conj()) / cell.nao
    g = B.Isdf(cell, B.ISDF_FP64)
    g.build_points(n_p, seed)
    g.fit_zeta(tau)
    g.coulomb_metric()
    K = torch.empty((cell.nkpts, cell.nao, cell.nao), dtype=torch.complex128, device="cuda")
    g.exchange(_dev(torch, P), K)
    torch.cuda.synchronize()
    _, _, V = o.fit(tau)
    Ko = O.exchange_matrix(o.X, V, P, cell.kmesh)
    assert np.abs(K.cpu().numpy() - Ko).max() < FP64_TOL


# ------------------------------------------------- grouped small fragments
def test_grouped_fragments_match_one_at_a_time(cuda, lib_built, c2):
    """Small fragments are contracted in groups (stacked rows, block-diagonal
    tiles).  The results equal those of each fragment contracted alone, and the
    oracle within the mixed tolerance; the tile-order autotuner changes only the
    order of the tiles."""
    from paper_2601_16379_gb300 import binding as B
    torch = cuda
    wl, o = c2
    frags = [W.make_fragment(wl.cell, wl.seed, i, n) for i, n in enumerate([5, 9, 14, 7, 11])]
    g = B.Isdf(wl.cell, B.ISDF_MIXED)
    g.build_points(wl.n_p, wl.seed)
    g.fit_zeta(1e-7)
    g.coulomb_metric()
    eris, ej, ek = gpu_eri(torch, g, frags, 1)
    for i, f in enumerate(frags):
        e1, j1, k1 = gpu_eri(torch, g, [f], 1)
        assert np.abs(e1[0] - eris[i]).max() < 1e-10
        assert abs(j1[0] - ej[i]) < 1e-10 and abs(k1[0] - ek[i]) < 1e-10
    for i in (0, 2):
        ref, (rj, rk) = o.eri(1e-7, frags[i])
        assert np.abs(eris[i] - ref).max() < MIXED_TOL
        assert abs(ej[i] - rj) < MIXED_TOL and abs(ek[i] - rk) < MIXED_TOL
    g.set_autotune(False)
    eris2, ej2, ek2 = gpu_eri(torch, g, frags, 1)
    for i in range(len(frags)):
        assert np.abs(eris2[i] - eris[i]).max() < 1e-10
    assert isinstance(g.autotune_report(), list)
    g.close()


def test_autotuned_tile_order_on_a_large_fragment(cuda, lib_built, c2):
    """A fragment with several waves of tiles triggers the tile-order tuning; the
    report names the chosen band, and the ERIs equal those without tuning."""
    from paper_2601_16379_gb300 import binding as B
    torch = cuda
    wl, o = c2
    f = W.make_fragment(wl.cell, wl.seed, 3, 40)   # n2 = 1600: 13 x 14 / 2 = 91 tiles per block
    big = W.make_fragment(wl.cell, wl.seed, 4, 72)  # n2 = 5184: 41 x 42 / 2 = 861 tiles
    res = []
    for tune in (True, False):
        g = B.Isdf(wl.cell, B.ISDF_MIXED)
        g.set_autotune(tune)
        g.build_points(wl.n_p, wl.seed)
        g.fit_zeta(1e-7)
        g.coulomb_metric()
        res.append(gpu_eri(torch, g, [f, big], 1))
        rep = g.autotune_report()
        if tune:
            assert any(e["tiles"] >= 861 and e["band"] in (6, 12, 24) for e in rep), rep
        else:
            assert rep == []
        g.close()
    for i in range(2):
        assert np.abs(res[0][0][i] - res[1][0][i]).max() < 1e-10
        assert abs(res[0][1][i] - res[1][1][i]) < 1e-10


@pytest.mark.parametrize("pipeline,band", [(0, 12), (1, 12), (1, 5)])
def test_tile_schedules_match_oracle(cuda, lib_built, c2, pipeline, band):
    """Each pipeline of the tensor-core tile kernel (K rows of 64 fp16 in 3
    stages, rows of 32 fp16 in 6 stages) and tile order gives the oracle's ERIs."""
    from paper_2601_16379_gb300 import binding as B
    torch = cuda
    wl, o = c2
    f = W.make_fragment(wl.cell, wl.seed, 4, 40)
    g = B.Isdf(wl.cell, B.ISDF_MIXED)
    g.set_tile_schedule(pipeline, band)
    g.build_points(wl.n_p, wl.seed)
    g.fit_zeta(1e-7)
    g.coulomb_metric()
    eris, ej, ek = gpu_eri(torch, g, [f], 1)
    ref, (rj, rk) = o.eri(1e-7, f)
    assert np.abs(eris[0] - ref).max() < MIXED_TOL
    assert abs(ej[0] - rj) < MIXED_TOL and abs(ek[0] - rk) < MIXED_TOL
    with pytest.raises(B.IsdfError):
        g.set_tile_schedule(2, 12)
    g.close()


@pytest.mark.parametrize("case", ["c1", "c2"])
def test_emulated_fit_gemm_matches_fp64(cuda, lib_built, c1, c2, case):
    """In the mixed path g^k = conj(X^k) Phi^k (Eq. 5) runs on the tensor cores with
    seven exact 7-bit slices per operand; eta^q then equals the FP64 path's to
    ~1e-14 relative, and the ranks of the factor of Pi^q are the same."""
    from paper_2601_16379_gb300 import binding as B
    torch = cuda
    wl, o = c1 if case == "c1" else c2
    s = {}
    for prec in (B.ISDF_FP64, B.ISDF_MIXED):
        g = B.Isdf(wl.cell, prec)
        g.build_points(wl.n_p, wl.seed)
        ranks = g.fit_zeta(1e-7)
        sz = g.sizes()
        eta = torch.empty((sz["nk"], sz["np"], sz["ng"]), dtype=torch.complex128, device="cuda")
        g.get(2, eta)
        s[prec] = (eta.cpu().numpy(), ranks)
        g.close()
    e64, em = s[B.ISDF_FP64][0], s[B.ISDF_MIXED][0]
    assert np.abs(em - e64).max() < 1e-12 * np.abs(e64).max()
    assert np.array_equal(s[B.ISDF_FP64][1], s[B.ISDF_MIXED][1])
    ref = o.eta
    assert np.abs(em - ref).max() < 1e-12 * np.abs(ref).max()


# ------------------------------------------- FP64-class tensor-core path
def test_fp64tc_eri_c1(cuda, lib_built, c1):
    """FP64_TC (float-float pair tensor, five- and four-slice exact tensor-core
    contractions) against the oracle at the FP64 tolerance, with a 7-orbital and a
    1-orbital fragment grouped with the workload's own."""
    from paper_2601_16379_gb300 import binding as B
    wl, o = c1
    tol = 1e-7
    frags = list(wl.fragments) + [W.make_fragment(wl.cell, wl.seed, 5, 7), W.make_fragment(wl.cell, wl.seed, 6, 1)]
    g = B.Isdf(wl.cell, B.ISDF_FP64_TC)
    g.build_points(wl.n_p, wl.seed)
    g.fit_zeta(tol)
    g.coulomb_metric()
    eris, ej, ek = gpu_eri(cuda, g, frags, 2)
    for i, f in enumerate(frags):
        ref, (rj, rk) = o.eri(tol, f)
        assert np.abs(eris[i] - ref).max() < FP64_TOL
        assert abs(ej[i] - rj) < FP64_TOL and abs(ek[i] - rk) < FP64_TOL
    g.close()


@pytest.mark.parametrize("limit", [1, 64 << 20])
def test_fp64tc_q_chunks_and_fp64_agreement(cuda, lib_built, c2, limit):
    """FP64_TC with the q-points of the sum split into chunks (the E' kernel then
    accumulates into its workspace across launches) on a 40-orbital fragment
    (several waves of tiles) and a small one: the ERIs agree with the FP64
    path's to 1e-9 Ha (an order below the FP64 tolerance, three below the mixed
    path's), and with the oracle within the FP64 tolerance."""
    from paper_2601_16379_gb300 import binding as B
    torch = cuda
    wl, o = c2
    frags = [W.make_fragment(wl.cell, wl.seed, 4, 40), W.make_fragment(wl.cell, wl.seed, 2, 9)]
    res = {}
    for prec in (B.ISDF_FP64, B.ISDF_FP64_TC):
        g = B.Isdf(wl.cell, prec)
        if prec == B.ISDF_FP64_TC:
            # slice workspace for one q-point per chunk (limit 1), or a few (~8 MB per q-point)
            g.set_workspace_limit(limit)
        g.build_points(wl.n_p, wl.seed)
        g.fit_zeta(1e-7)
        g.coulomb_metric()
        res[prec] = gpu_eri(torch, g, frags, prec)
        g.close()
    d, t = res[B.ISDF_FP64], res[B.ISDF_FP64_TC]
    for i in range(len(frags)):
        assert np.abs(t[0][i] - d[0][i]).max() < 1e-9
        assert abs(t[1][i] - d[1][i]) < 1e-9 and abs(t[2][i] - d[2][i]) < 1e-9
    ref, (rj, rk) = o.eri(1e-7, frags[1])
    assert np.abs(t[0][1] - ref).max() < FP64_TOL
    assert abs(t[1][1] - rj) < FP64_TOL and abs(t[2][1] - rk) < FP64_TOL

