"""ctypes binding of libisdf (include/isdf.h).

Argument marshalling only: every step of the k-ISDF path runs in the CUDA
library.  Device buffers are passed as raw pointers (``tensor.data_ptr()`` of
PyTorch CUDA tensors, which supply memory and streams).  There is no CPU
fallback: if ``libisdf.so`` is missing or cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as ct
from pathlib import Path
from typing import List, Optional, Sequence

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libisdf.so"

ISDF_FP64 = 0
ISDF_MIXED = 1
ISDF_FP64_TC = 2

STATUS = {0: "ISDF_OK", -1: "ISDF_ERR_ARG", -2: "ISDF_ERR_OOM", -3: "ISDF_ERR_CUDA",
          -4: "ISDF_ERR_NUMERIC", -5: "ISDF_ERR_TIMEOUT", -6: "ISDF_ERR_STATE"}

# Every entry point declared in include/isdf.h.
EXPORTS = ["isdf_create", "isdf_build_points", "isdf_set_points", "isdf_fit_zeta",
           "isdf_coulomb_metric", "isdf_coulomb_metric_eta", "isdf_fragment_eri", "isdf_exchange",
           "isdf_ao_eri", "isdf_sos_polarizability",
           "isdf_set_time_reversal", "isdf_set_workspace_limit", "isdf_set_autotune", "isdf_autotune_report",
           "isdf_set_tile_schedule",
           "isdf_get", "isdf_sizes",
           "isdf_launch_count", "isdf_timing_enable", "isdf_timing_get", "isdf_eri_traces_noalloc",
           "isdf_last_error", "isdf_destroy"]


class IsdfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class CellDesc(ct.Structure):
    _fields_ = [("lattice", ct.c_double * 9), ("natm", ct.c_int), ("coords", ct.POINTER(ct.c_double)),
                ("nshell", ct.c_int), ("shell_atom", ct.POINTER(ct.c_int)), ("shell_l", ct.POINTER(ct.c_int)),
                ("shell_nprim", ct.POINTER(ct.c_int)), ("exps", ct.POINTER(ct.c_double)),
                ("coefs", ct.POINTER(ct.c_double)), ("kmesh", ct.c_int * 3), ("mesh", ct.c_int * 3),
                ("lattice_eps", ct.c_double)]


_lib = None


def load(path: Optional[str] = None) -> ct.CDLL:
    """Load libisdf.so (raises if it is absent: the CUDA path is the only path)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise RuntimeError(f"libisdf.so not built ({p}); run __graft_entry__.build()")
    lib = ct.CDLL(str(p))
    vp, i32p, dp = ct.c_void_p, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_double)
    lib.isdf_create.argtypes = [ct.POINTER(CellDesc), ct.c_int, vp, ct.POINTER(vp)]
    lib.isdf_build_points.argtypes = [vp, ct.c_int, ct.c_uint64, ct.c_double, i32p]
    lib.isdf_set_points.argtypes = [vp, ct.c_int, i32p]
    lib.isdf_fit_zeta.argtypes = [vp, ct.c_double, i32p]
    lib.isdf_coulomb_metric.argtypes = [vp, vp]
    lib.isdf_coulomb_metric_eta.argtypes = [vp, vp]
    lib.isdf_fragment_eri.argtypes = [vp, ct.c_int, i32p, ct.POINTER(vp), ct.POINTER(vp), ct.POINTER(vp), dp, dp]
    lib.isdf_exchange.argtypes = [vp, vp, vp]
    lib.isdf_ao_eri.argtypes = [vp, ct.c_int, i32p, vp]
    lib.isdf_sos_polarizability.argtypes = [vp, vp, ct.c_int, ct.c_int, dp, ct.c_double, vp, dp]
    lib.isdf_set_time_reversal.argtypes = [vp, ct.c_int]
    lib.isdf_set_workspace_limit.argtypes = [vp, ct.c_uint64]
    lib.isdf_set_autotune.argtypes = [vp, ct.c_int]
    lib.isdf_autotune_report.argtypes = [vp, ct.c_char_p, ct.c_size_t]
    lib.isdf_set_tile_schedule.argtypes = [vp, ct.c_int, ct.c_int]
    lib.isdf_get.argtypes = [vp, ct.c_int, vp]
    lib.isdf_sizes.argtypes = [vp, ct.POINTER(ct.c_int64)]
    lib.isdf_launch_count.argtypes = [vp]
    lib.isdf_launch_count.restype = ct.c_int64
    lib.isdf_timing_enable.argtypes = [vp, ct.c_int]
    lib.isdf_timing_get.argtypes = [vp, ct.c_int, dp, ct.POINTER(ct.c_int64), dp]
    lib.isdf_eri_traces_noalloc.argtypes = [vp, ct.c_int, vp, dp, dp, vp]
    lib.isdf_last_error.argtypes = [vp]
    lib.isdf_last_error.restype = ct.c_char_p
    lib.isdf_destroy.argtypes = [vp]
    lib.isdf_destroy.restype = None
    for name in EXPORTS:
        if name not in ("isdf_launch_count", "isdf_last_error", "isdf_destroy"):
            getattr(lib, name).restype = ct.c_int
    if path is None:
        _lib = lib
    return lib


def _ptr(x) -> ct.c_void_p:
    if x is None:
        return ct.c_void_p(0)
    if isinstance(x, int):
        return ct.c_void_p(x)
    return ct.c_void_p(x.data_ptr())


class Isdf:
    """One handle of the library for a cell (see include/isdf.h for each call)."""

    def __init__(self, cell, precision: int = ISDF_FP64, stream=None, lattice_eps: float = 0.0):
        self.lib = load()
        self._keep = []
        d = CellDesc()
        d.lattice[:] = [float(x) for x in np.asarray(cell.lattice, np.float64).reshape(9)]
        coords = np.ascontiguousarray(cell.coords, np.float64).reshape(-1)
        atoms = np.array([s.atom for s in cell.shells], np.int32)
        ls = np.array([s.l for s in cell.shells], np.int32)
        nprim = np.array([len(s.exps) for s in cell.shells], np.int32)
        exps = np.array([e for s in cell.shells for e in s.exps], np.float64)
        coefs = np.array([c for s in cell.shells for c in s.coefs], np.float64)
        self._keep += [coords, atoms, ls, nprim, exps, coefs]
        d.natm = coords.size // 3
        d.coords = coords.ctypes.data_as(ct.POINTER(ct.c_double))
        d.nshell = len(cell.shells)
        d.shell_atom = atoms.ctypes.data_as(ct.POINTER(ct.c_int))
        d.shell_l = ls.ctypes.data_as(ct.POINTER(ct.c_int))
        d.shell_nprim = nprim.ctypes.data_as(ct.POINTER(ct.c_int))
        d.exps = exps.ctypes.data_as(ct.POINTER(ct.c_double))
        d.coefs = coefs.ctypes.data_as(ct.POINTER(ct.c_double))
        d.kmesh[:] = list(cell.kmesh)
        d.mesh[:] = list(cell.mesh)
        d.lattice_eps = float(lattice_eps)
        self.precision = precision
        h = ct.c_void_p()
        st = ct.c_void_p(0 if stream is None else int(getattr(stream, "cuda_stream", stream)))
        rc = self.lib.isdf_create(ct.byref(d), int(precision), st, ct.byref(h))
        if rc != 0:
            raise IsdfError(rc, "isdf_create failed")
        self.h = h

    # -- helpers -----------------------------------------------------------
    def _check(self, rc: int):
        if rc != 0:
            raise IsdfError(rc, self.lib.isdf_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.isdf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sizes(self):
        out = (ct.c_int64 * 4)()
        self._check(self.lib.isdf_sizes(self.h, out))
        return dict(nao=out[0], nk=out[1], ng=out[2], np=out[3])

    def launch_count(self) -> int:
        return int(self.lib.isdf_launch_count(self.h))

    def timing(self, enable: bool):
        self._check(self.lib.isdf_timing_enable(self.h, 1 if enable else 0))

    def set_time_reversal(self, enable: bool):
        """Pair q with -q in the fragment contraction (default on)."""
        self._check(self.lib.isdf_set_time_reversal(self.h, 1 if enable else 0))

    def set_workspace_limit(self, nbytes: int):
        """Device bytes for one q-chunk of the fp16 slices of the mixed contraction."""
        self._check(self.lib.isdf_set_workspace_limit(self.h, ct.c_uint64(int(nbytes))))

    def set_autotune(self, enable: bool):
        """Tile-order tuning of the mixed contraction (default on)."""
        self._check(self.lib.isdf_set_autotune(self.h, 1 if enable else 0))

    def set_tile_schedule(self, pipeline: int, band: int):
        """Fix the tile schedule of the mixed contraction (turns tuning off)."""
        self._check(self.lib.isdf_set_tile_schedule(self.h, int(pipeline), int(band)))

    def autotune_report(self):
        """The tile-order choices made so far, as a list of dicts."""
        import json
        buf = ct.create_string_buffer(1 << 16)
        self._check(self.lib.isdf_autotune_report(self.h, buf, len(buf)))
        return json.loads(buf.value.decode())

    def stage_time(self, stage: int):
        """(device ms summed, launches, algorithmic flops summed) of a stage."""
        ms, n, fl = ct.c_double(), ct.c_int64(), ct.c_double()
        self._check(self.lib.isdf_timing_get(self.h, int(stage), ct.byref(ms), ct.byref(n), ct.byref(fl)))
        return ms.value, n.value, fl.value

    # -- the four steps ----------------------------------------------------
    def build_points(self, n_p: int, seed: int, chol_tol: float = 1e-14) -> np.ndarray:
        ips = np.zeros(n_p, np.int32)
        self._check(self.lib.isdf_build_points(self.h, int(n_p), ct.c_uint64(int(seed) & (2**64 - 1)),
                                               float(chol_tol), ips.ctypes.data_as(ct.POINTER(ct.c_int32))))
        return ips

    def set_points(self, ips: Sequence[int]):
        a = np.ascontiguousarray(np.asarray(ips, np.int32))
        self._check(self.lib.isdf_set_points(self.h, int(a.size), a.ctypes.data_as(ct.POINTER(ct.c_int32))))

    def fit_zeta(self, solve_tol: float) -> np.ndarray:
        nk = self.sizes()["nk"]
        ranks = np.zeros(nk, np.int32)
        self._check(self.lib.isdf_fit_zeta(self.h, float(solve_tol), ranks.ctypes.data_as(ct.POINTER(ct.c_int32))))
        return ranks

    def coulomb_metric(self, V_out=None):
        self._check(self.lib.isdf_coulomb_metric(self.h, _ptr(V_out)))

    def coulomb_metric_eta(self, V_out=None):
        """The Coulomb kernel by Eqs. 7-8 (from eta, zeta never formed)."""
        self._check(self.lib.isdf_coulomb_metric_eta(self.h, _ptr(V_out)))

    def fragment_eri(self, C_list: List, gamma_list: Optional[List] = None, eri_out: Optional[List] = None,
                     traces: bool = True):
        n = len(C_list)
        norb = np.array([int(c.shape[-1]) for c in C_list], np.int32)
        Cp = (ct.c_void_p * max(n, 1))(*[_ptr(c) for c in C_list])
        gp = None
        if gamma_list is not None:
            gp = (ct.c_void_p * max(n, 1))(*[_ptr(g) for g in gamma_list])
        ep = None
        if eri_out is not None:
            ep = (ct.c_void_p * max(n, 1))(*[_ptr(e) for e in eri_out])
        ej = np.zeros(max(n, 1), np.float64)
        ek = np.zeros(max(n, 1), np.float64)
        dp = ct.POINTER(ct.c_double)
        self._check(self.lib.isdf_fragment_eri(
            self.h, n, norb.ctypes.data_as(ct.POINTER(ct.c_int32)), Cp, gp, ep,
            ej.ctypes.data_as(dp) if traces else None, ek.ctypes.data_as(dp) if traces else None))
        return ej[:n], ek[:n]

    def exchange(self, P, K_out):
        """k-point exchange matrix K^k (Eq. 10) for the AO density matrices P^k."""
        self._check(self.lib.isdf_exchange(self.h, _ptr(P), _ptr(K_out)))
        return K_out

    def ao_eri(self, quartets, out):
        """AO-level integrals (mu k1 nu k2|lam k3 sig k4) for k-quartets (Eq. 9), FP64."""
        q = np.ascontiguousarray(np.asarray(quartets, np.int32).reshape(-1, 4))
        self._check(self.lib.isdf_ao_eri(self.h, int(q.shape[0]), q.ctypes.data_as(ct.POINTER(ct.c_int32)),
                                         _ptr(out)))
        return out

    def sos_polarizability(self, C, eps, n_occ: int, tau: float, chi_out=None) -> float:
        """k-SOS-MP2 polarisability chi^Q(tau) (into chi_out, if given) and S(tau) (Eqs. 11-15)."""
        e = np.ascontiguousarray(np.asarray(eps, np.float64))
        s = ct.c_double()
        self._check(self.lib.isdf_sos_polarizability(
            self.h, _ptr(C), int(C.shape[-1]), int(n_occ), e.ctypes.data_as(ct.POINTER(ct.c_double)),
            float(tau), _ptr(chi_out), ct.byref(s)))
        return s.value

    def get(self, what: int, out):
        self._check(self.lib.isdf_get(self.h, int(what), _ptr(out)))
        return out


def eri_traces_noalloc(eri, n_orb: int, gamma, stream=None):
    """E_J, E_K of one fragment from its chemist-order ERIs, through the
    allocation-free entry point (no handle, no device allocation)."""
    lib = load()
    ej, ek = ct.c_double(), ct.c_double()
    st = ct.c_void_p(0 if stream is None else int(getattr(stream, "cuda_stream", stream)))
    rc = lib.isdf_eri_traces_noalloc(_ptr(eri), int(n_orb), _ptr(gamma), ct.byref(ej), ct.byref(ek), st)
    if rc != 0:
        raise IsdfError(rc, lib.isdf_last_error(None).decode())
    return ej.value, ek.value
