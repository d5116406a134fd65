"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/isdf.h declares.  No compute calls (no GPU needed)."""
import ctypes
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def declared_symbols():
    text = (ROOT / "include" / "isdf.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(isdf_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_steps():
    syms = declared_symbols()
    for s in ("isdf_create", "isdf_build_points", "isdf_fit_zeta", "isdf_coulomb_metric",
              "isdf_fragment_eri", "isdf_destroy", "isdf_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib_built):
    lib = ctypes.CDLL(str(lib_built))
    for s in declared_symbols():
        assert hasattr(lib, s), f"{s} declared in include/isdf.h but not exported"


def test_binding_lists_match_header(lib_built):
    from paper_2601_16379_gb300 import binding
    assert sorted(binding.EXPORTS) == declared_symbols()
    binding.load()


def test_library_is_sm_103a(lib_built):
    from paper_2601_16379_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_product_path_does_not_import_oracle():
    pkg = ROOT / "paper_2601_16379_gb300"
    for p in list(pkg.rglob("*.py")) + list(pkg.rglob("*.cu")) + list(pkg.rglob("*.cuh")):
        src = p.read_text()
        assert "import oracle" not in src and "from oracle" not in src, p
