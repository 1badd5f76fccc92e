"""The C-ABI library builds, loads without a GPU, and exports every function
its public header declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(admm_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2110_06879_gb300 import admm
    lib = ctypes.CDLL(admm.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 19
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_defaults_and_status_strings_without_gpu():
    from paper_2110_06879_gb300 import admm
    o = admm.default_options()
    assert o.rho_pq == 10.0 and o.rho_va == 1000.0 and o.max_outer == 20 and o.max_inner == 1000
    assert o.line_limit_frac == 0.99 and o.two_level == 1
    assert admm.lib().admm_status_string(0) == b"ADMM_OK"
    assert admm.lib().admm_status_string(-3) == b"ADMM_ERR_NUMERICAL"
