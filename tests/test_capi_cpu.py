"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "wbfbt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wbfbt_[a-zA-Z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_1607_03936_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert len(syms) >= 17
    for s in syms:
        assert hasattr(lib, s), s


def test_binding_symbol_list_matches_header():
    from paper_1607_03936_gb300 import wbfbt
    assert sorted(wbfbt.SYMBOLS) == declared_symbols()


def test_status_strings_and_defaults_without_gpu():
    from paper_1607_03936_gb300 import wbfbt
    lib = wbfbt.lib()
    assert lib.wbfbt_status_string(0) == b"ok"
    assert b"iteration" in lib.wbfbt_status_string(-5)
    o = wbfbt.default_opts()
    assert (o.a_l, o.a_r, o.restart, o.cheb_degree, o.mg_min_n, o.precision, o.schur_sign, o.use_graphs,
            o.elem_kernels) == (1.0, 0.0, 50, 3, 4, 0, -1, 1, 0)
    # argument validation happens before any device call
    m = wbfbt.Mesh(2, 2, 2, 1.0, 1.0, 1.0)
    h = ctypes.c_void_p()
    assert lib.wbfbt_create(ctypes.byref(m), 9, ctypes.c_void_p(1), None, None, ctypes.byref(h)) == -1
    assert lib.wbfbt_apply_A(None, None, None, 0) == -1
    assert lib.wbfbt_set_geometry(None, None) == -1
    assert lib.wbfbt_node_coords(ctypes.byref(m), 2, None, None) == -1
    assert lib.wbfbt_sinker_setup_at(ctypes.byref(m), 2, None, None, 0, 0.1, 200.0, 1e4, 10.0, None, None,
                                     None) == -1
    assert lib.wbfbt_load_learned(None, b"net.bin") == -1
    assert lib.wbfbt_train_learned(None, None, b"net.bin") == -1
    # options out of range are rejected before any device call
    for field, value in (("elem_kernels", 3), ("elem_kernels", -1), ("restart", 0), ("cheb_degree", 17),
                         ("precision", 2), ("mg_min_n", 0)):
        bad = wbfbt.default_opts()
        setattr(bad, field, value)
        assert lib.wbfbt_create(ctypes.byref(m), 2, ctypes.c_void_p(1), ctypes.byref(bad), None,
                                ctypes.byref(h)) == -1, field
