"""Seeded synthetic workloads for the k-ISDF fragment-ERI path.

This module only *generates inputs*: cell geometry, Cartesian Gaussian shells,
k-mesh and grid sizes, interpolation-point counts, fragment coefficient
matrices C^k_{mu p} and fragment density matrices gamma.  It holds none of the
method's arithmetic (no orbital evaluation, fitting, Coulomb or ERI work), so
that both the CUDA path and the FP64 oracle can consume the same inputs without
sharing any of the computation.

The five named workloads follow the paper's setting (Section II, Eq. 1 and
Eq. 17; Table I gives the diamond shape N_AO = 26 that c2/c4/c5 mimic):

====  ==========================================  ====  ====  ====  ======================
name  cell / basis                                 Nk    grid  N_P   fragments
====  ==========================================  ====  ====  ====  ======================
c1    a=6.0, 2 atoms, s(0.5)+p(1.5): 8 AOs         2^3   16^3  64    1 x 4
c2    a=6.0, 2 atoms, s,p,p,d(cart): 26 AOs        3^3   24^3  200   1 x 40
c3    a=7.5, 4 fcc atoms, 13 AOs each: 52 AOs      4^3   32^3  500   3 x 60
c4    as c2                                        6^3   24^3  300   40, n_f ~ U[20,120]
c5    as c2                                        10^3  24^3  300   64, n_f ~ U[40,200]
====  ==========================================  ====  ====  ====  ======================

Random numbers: every stream is ``numpy.random.default_rng([seed, tag])`` with
the workload seed ``20260000 + config number`` and a fixed integer tag per
quantity, so each array can be regenerated independently.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Tags of the independent random streams.
TAG_MO = 1
TAG_U = 2
TAG_GAMMA = 3
TAG_SIZES = 4
TAG_REAL = 5
TAG_SINGLEK = 6
TAG_EPS = 7
TAG_POINTS = 8

SEED_BASE = 20260000


@dataclass(frozen=True)
class Shell:
    """One Cartesian Gaussian shell (contraction of normalised primitives)."""
    atom: int
    l: int
    exps: Tuple[float, ...]
    coefs: Tuple[float, ...]

    @property
    def ncart(self) -> int:
        return (self.l + 1) * (self.l + 2) // 2


@dataclass
class Cell:
    """Unit cell, basis and sampling (paper Eq. 1 and Section II)."""
    lattice: np.ndarray          # (3, 3) float64, rows are a_1, a_2, a_3 in Bohr
    coords: np.ndarray           # (natm, 3) float64, Bohr
    shells: List[Shell]
    kmesh: Tuple[int, int, int]  # Gamma-centred mesh n_k per axis
    mesh: Tuple[int, int, int]   # real-space grid points per axis

    @property
    def nao(self) -> int:
        return sum(s.ncart for s in self.shells)

    @property
    def nkpts(self) -> int:
        return int(np.prod(self.kmesh))

    @property
    def ngrid(self) -> int:
        return int(np.prod(self.mesh))

    @property
    def volume(self) -> float:
        return float(abs(np.linalg.det(self.lattice)))


@dataclass
class Fragment:
    """Fragment orbitals phi_p = Nk^{-1/2} sum_k sum_mu C^k_{mu p} phi^k_mu (Eq. 17)."""
    C: np.ndarray       # (Nk, N_AO, n_f) complex128
    gamma: np.ndarray   # (n_f, n_f) complex128 Hermitian, eigenvalues in {0, 2}

    @property
    def norb(self) -> int:
        return int(self.C.shape[2])


@dataclass
class Workload:
    name: str
    cell: Cell
    n_p: int
    seed: int
    frag_sizes: List[int]
    chol_tol: float = 1e-14     # relative stop of the interpolation-point pivoted Cholesky
    solve_tol: float = 1e-12    # relative truncation of the Pi^q pivoted Cholesky
    description: str = ""
    fragments: Optional[List[Fragment]] = field(default=None, repr=False)


# ----------------------------------------------------------------------------
# Basis sets used by the named workloads
# ----------------------------------------------------------------------------

def _shells_sp(natm: int) -> List[Shell]:
    out = []
    for a in range(natm):
        out.append(Shell(a, 0, (0.5,), (1.0,)))
        out.append(Shell(a, 1, (1.5,), (1.0,)))
    return out


def _shells_spd13(natm: int) -> List[Shell]:
    out = []
    for a in range(natm):
        out.append(Shell(a, 0, (0.5,), (1.0,)))
        out.append(Shell(a, 1, (0.5,), (1.0,)))
        out.append(Shell(a, 1, (1.5,), (1.0,)))
        out.append(Shell(a, 2, (1.0,), (1.0,)))
    return out


def cubic_cell(a: float, frac_coords: Sequence[Sequence[float]], shells: List[Shell],
               kmesh: Tuple[int, int, int], mesh: Tuple[int, int, int]) -> Cell:
    lat = np.eye(3) * float(a)
    coords = np.asarray(frac_coords, dtype=np.float64) @ lat
    return Cell(lat, coords, shells, tuple(int(x) for x in kmesh), tuple(int(x) for x in mesh))


# ----------------------------------------------------------------------------
# Random inputs
# ----------------------------------------------------------------------------

def _rng(seed: int, tag: int, extra: int = 0) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(tag), int(extra)])


def _cgauss(rng: np.random.Generator, shape) -> np.ndarray:
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * np.sqrt(0.5)


def _qr_pos(a: np.ndarray) -> np.ndarray:
    """Reduced QR with the phases fixed so that diag(R) is real positive."""
    q, r = np.linalg.qr(a)
    d = np.diagonal(r).copy()
    ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1.0), 1.0)
    return q * ph[None, :]


def mo_coefficients(cell: Cell, seed: int) -> np.ndarray:
    """Seeded random MO coefficients, orthonormal per k (identity metric)."""
    nk, nao = cell.nkpts, cell.nao
    rng = _rng(seed, TAG_MO)
    g = _cgauss(rng, (nk, nao, nao))
    return np.stack([_qr_pos(g[k]) for k in range(nk)])


def orbital_energies(cell: Cell, seed: int, n_occ: int) -> np.ndarray:
    """Seeded synthetic orbital energies per k (Ha), ascending, the first n_occ
    occupied in [-1.0, -0.2] and the rest virtual in [0.2, 2.0] (a gap around
    the chemical potential 0), shape (Nk, N_AO).  Stand-ins for k-HF energies."""
    nk, nao = cell.nkpts, cell.nao
    rng = _rng(seed, TAG_EPS)
    occ = np.sort(rng.uniform(-1.0, -0.2, size=(nk, n_occ)), axis=1)
    vir = np.sort(rng.uniform(0.2, 2.0, size=(nk, nao - n_occ)), axis=1)
    return np.concatenate([occ, vir], axis=1)


def seeded_points(cell: Cell, n_p: int, seed: int) -> np.ndarray:
    """n_p distinct grid indices drawn uniformly (a seeded stand-in for the
    interpolation points, given to both sides when the selection itself is
    not what a test compares)."""
    if n_p > cell.ngrid:
        raise ValueError("more points than grid points")
    return np.sort(_rng(seed, TAG_POINTS).choice(cell.ngrid, size=n_p, replace=False)).astype(np.int32)


def make_fragment(cell: Cell, seed: int, index: int, norb: int,
                  mo: Optional[np.ndarray] = None) -> Fragment:
    """Fragment of `norb` orbitals: a seeded random isometry of the Bloch MOs."""
    nk, nao = cell.nkpts, cell.nao
    if norb > nk * nao:
        raise ValueError("fragment larger than the supercell orbital space")
    if mo is None:
        mo = mo_coefficients(cell, seed)
    u = _qr_pos(_cgauss(_rng(seed, TAG_U, index), (nk * nao, norb))).reshape(nk, nao, norb)
    C = np.einsum("kmn,knp->kmp", mo, u)
    w = _qr_pos(_cgauss(_rng(seed, TAG_GAMMA, index), (norb, norb)))[:, : norb // 2]
    gamma = 2.0 * (w @ w.conj().T)
    gamma = 0.5 * (gamma + gamma.conj().T)
    return Fragment(np.ascontiguousarray(C), np.ascontiguousarray(gamma))


def kpoint_index(m: Sequence[int], kmesh: Sequence[int]) -> int:
    """Flat index of k-mesh point m (row-major, last axis fastest)."""
    return (int(m[0]) % kmesh[0]) * kmesh[1] * kmesh[2] + (int(m[1]) % kmesh[1]) * kmesh[2] + (int(m[2]) % kmesh[2])


def make_real_fragment(cell: Cell, seed: int, norb: int) -> Fragment:
    """Fragment whose orbitals are real in the supercell: C^{-k} = conj(C^k)."""
    nk, nao = cell.nkpts, cell.nao
    rng = _rng(seed, TAG_REAL)
    C = np.zeros((nk, nao, norb), np.complex128)
    km = cell.kmesh
    for m0 in range(km[0]):
        for m1 in range(km[1]):
            for m2 in range(km[2]):
                k = kpoint_index((m0, m1, m2), km)
                kn = kpoint_index((-m0, -m1, -m2), km)
                if k < kn:
                    C[k] = _cgauss(rng, (nao, norb))
                    C[kn] = C[k].conj()
                elif k == kn:
                    C[k] = rng.standard_normal((nao, norb))
    C /= np.sqrt(nk * nao)
    w = np.linalg.qr(rng.standard_normal((norb, norb)))[0][:, : norb // 2]
    gamma = (2.0 * (w @ w.T)).astype(np.complex128)
    return Fragment(C, gamma)


def make_singlek_fragment(cell: Cell, seed: int, norb: int) -> Tuple[Fragment, np.ndarray]:
    """Fragment whose orbital p has C^k nonzero for a single k_p only.

    Returns the fragment and the k index of each orbital.
    """
    nk, nao = cell.nkpts, cell.nao
    rng = _rng(seed, TAG_SINGLEK)
    kp = rng.integers(0, nk, size=norb)
    C = np.zeros((nk, nao, norb), np.complex128)
    for p in range(norb):
        v = _cgauss(rng, nao)
        C[kp[p], :, p] = v / np.linalg.norm(v)
    gamma = np.eye(norb, dtype=np.complex128)
    return Fragment(C, gamma), kp


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

BCC2 = [[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]]
FCC4 = [[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]]

_SPECS = {
    "c1": dict(a=6.0, atoms=BCC2, basis="sp", kmesh=2, mesh=16, n_p=64, frags=("fixed", 1, 4),
               description="Nk=2^3, 16^3 grid, 8 AOs, N_P=64, 1 fragment x 4, complex128"),
    "c2": dict(a=6.0, atoms=BCC2, basis="spd13", kmesh=3, mesh=24, n_p=200, frags=("fixed", 1, 40),
               description="Nk=3^3, 24^3 grid, 26 AOs, N_P=200, 1 fragment x 40, complex128"),
    "c3": dict(a=7.5, atoms=FCC4, basis="spd13", kmesh=4, mesh=32, n_p=500, frags=("fixed", 3, 60),
               description="Nk=4^3, 32^3 grid, 52 AOs, N_P=500, 3 fragments x 60, mixed"),
    "c4": dict(a=6.0, atoms=BCC2, basis="spd13", kmesh=6, mesh=24, n_p=300, frags=("uniform", 40, 20, 120),
               description="Nk=6^3, 24^3 grid, 26 AOs, N_P=300, 40 fragments n_f~U[20,120]"),
    "c5": dict(a=6.0, atoms=BCC2, basis="spd13", kmesh=10, mesh=24, n_p=300, frags=("uniform", 64, 40, 200),
               description="Nk=10^3, 24^3 grid, 26 AOs, N_P=300, 64 fragments n_f~U[40,200]"),
}

CONFIG_NUMBER = {"c1": 1, "c2": 2, "c3": 3, "c4": 4, "c5": 5}


def workload(name: str, *, kmesh: Optional[int] = None, mesh: Optional[int] = None,
             n_p: Optional[int] = None, frag_sizes: Optional[List[int]] = None,
             with_fragments: bool = True) -> Workload:
    """Build a named workload; keyword overrides give the reduced variants used by tests."""
    spec = _SPECS[name]
    natm = len(spec["atoms"])
    shells = _shells_sp(natm) if spec["basis"] == "sp" else _shells_spd13(natm)
    km = spec["kmesh"] if kmesh is None else kmesh
    gm = spec["mesh"] if mesh is None else mesh
    cell = cubic_cell(spec["a"], spec["atoms"], shells, (km, km, km), (gm, gm, gm))
    seed = SEED_BASE + CONFIG_NUMBER[name]
    if frag_sizes is None:
        fr = spec["frags"]
        if fr[0] == "fixed":
            frag_sizes = [fr[2]] * fr[1]
        else:
            frag_sizes = [int(x) for x in _rng(seed, TAG_SIZES).integers(fr[2], fr[3], size=fr[1], endpoint=True)]
    wl = Workload(name=name, cell=cell, n_p=spec["n_p"] if n_p is None else n_p, seed=seed,
                  frag_sizes=list(frag_sizes), description=spec["description"])
    if with_fragments:
        wl.fragments = make_fragments(wl)
    return wl


def make_fragments(wl: Workload, indices: Optional[Sequence[int]] = None) -> List[Fragment]:
    mo = mo_coefficients(wl.cell, wl.seed)
    idx = range(len(wl.frag_sizes)) if indices is None else indices
    return [make_fragment(wl.cell, wl.seed, i, wl.frag_sizes[i], mo) for i in idx]


def custom_cell(a: float, frac_coords, shells: List[Shell], kmesh, mesh) -> Cell:
    km = (kmesh,) * 3 if np.isscalar(kmesh) else tuple(kmesh)
    gm = (mesh,) * 3 if np.isscalar(mesh) else tuple(mesh)
    return cubic_cell(a, frac_coords, shells, km, gm)
