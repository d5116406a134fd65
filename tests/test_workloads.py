"""The seeded input generator: determinism, shapes and the stated properties."""
import numpy as np

from paper_2601_16379_gb300 import workloads as W


def test_named_workload_shapes():
    for name, nao, nk, ng, n_p in (("c1", 8, 8, 4096, 64), ("c2", 26, 27, 13824, 200),
                                   ("c3", 52, 64, 32768, 500), ("c4", 26, 216, 13824, 300),
                                   ("c5", 26, 1000, 13824, 300)):
        wl = W.workload(name, with_fragments=False)
        assert (wl.cell.nao, wl.cell.nkpts, wl.cell.ngrid, wl.n_p) == (nao, nk, ng, n_p)
    c4 = W.workload("c4", with_fragments=False)
    assert len(c4.frag_sizes) == 40 and min(c4.frag_sizes) >= 20 and max(c4.frag_sizes) <= 120
    c5 = W.workload("c5", with_fragments=False)
    assert len(c5.frag_sizes) == 64 and min(c5.frag_sizes) >= 40 and max(c5.frag_sizes) <= 200


def test_seeded_and_deterministic():
    a = W.workload("c2")
    b = W.workload("c2")
    assert np.array_equal(a.fragments[0].C, b.fragments[0].C)
    assert W.workload("c4", with_fragments=False).frag_sizes == W.workload("c4", with_fragments=False).frag_sizes


def test_fragment_is_isometry_and_gamma_projector():
    wl = W.workload("c1")
    f = wl.fragments[0]
    U = f.C.reshape(-1, f.norb)   # stacked (k, mu) rows; MOs unitary per k -> isometry
    assert np.allclose(U.conj().T @ U, np.eye(f.norb), atol=1e-12)
    ev = np.linalg.eigvalsh(f.gamma)
    assert np.allclose(f.gamma, f.gamma.conj().T)
    assert np.allclose(np.sort(ev), [0.0] * (f.norb - f.norb // 2) + [2.0] * (f.norb // 2), atol=1e-12)


def test_real_and_singlek_fragments():
    cell = W.workload("c1", with_fragments=False).cell
    f = W.make_real_fragment(cell, 3, 5)
    km = np.array([W.kpoint_index((-m0, -m1, -m2), cell.kmesh)
                   for m0 in range(2) for m1 in range(2) for m2 in range(2)])
    assert np.allclose(f.C[km], f.C.conj())
    g, kp = W.make_singlek_fragment(cell, 3, 6)
    for p in range(6):
        nz = np.nonzero(np.abs(g.C[:, :, p]).sum(axis=1))[0]
        assert list(nz) == [kp[p]]


def test_orbital_energies_seeded_with_a_gap():
    wl = W.workload("c1", with_fragments=False)
    e1 = W.orbital_energies(wl.cell, 5, 3)
    e2 = W.orbital_energies(wl.cell, 5, 3)
    assert np.array_equal(e1, e2)
    assert e1.shape == (wl.cell.nkpts, wl.cell.nao)
    assert (e1[:, :3] <= -0.2).all() and (e1[:, 3:] >= 0.2).all()
    assert (np.diff(e1[:, :3], axis=1) >= 0).all() and (np.diff(e1[:, 3:], axis=1) >= 0).all()
