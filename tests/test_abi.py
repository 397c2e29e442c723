"""The C-ABI library builds, loads and exports every entry point of include/*.h.

No compute call is made here (these run without a GPU)."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\**\s+\**(sc4dvar_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_path_entry_points():
    names = declared_symbols()
    for must in ("sc4dvar_fwd", "sc4dvar_gn_hessian_apply_block", "sc4dvar_build_precond",
                 "sc4dvar_pcg", "sc4dvar_gauss_newton", "sc4dvar_tlm_block", "sc4dvar_adj_block",
                 "sc4dvar_gradient", "sc4dvar_precond_apply", "sc4dvar_kappa_estimate"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import ctypes

    from paper_2401_15758_gb300 import _abi, build
    build.build()
    lib = ctypes.CDLL(build.LIB)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert declared_symbols() <= set(_abi.SIGNATURES), declared_symbols() - set(_abi.SIGNATURES)


def test_binding_loads_without_gpu():
    import paper_2401_15758_gb300 as g
    assert g.lib.sc4dvar_version() >= 100
