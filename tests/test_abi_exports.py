"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/pair.h declares (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            syms += re.findall(r"^PAIR_API\s+[\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M)
    return syms


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ("air_setup", "air_vcycle", "air_solve", "air_free", "si_solve", "dg_assemble_hex",
              "pair_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    from paper_1910_11463_gb300 import build as B
    B.build()
    lib = ctypes.CDLL(B.LIB)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_defaults_callable_without_gpu():
    from paper_1910_11463_gb300 import pair
    p = pair.default_air_params()
    assert (p.distance, p.theta, p.eps_R, p.max_coarse, p.coarse_sweeps, p.precision) == (1, 0.25, 0.01, 100, 20, 1)
    s = pair.default_si_params()
    assert s.tol == 1e-8 and s.use_graphs == 1
