"""The C ABI: the in-tree library builds, loads and exports every entry
point declared in include/*.h; host-side argument checks need no GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2506_08355_gb300 import build as B
from paper_2506_08355_gb300 import lrep

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    pat = re.compile(r"^\s*(?:lrep_status|void|int64_t|const\s+char\s*\*)\s*(lrep_\w+)\s*\(", re.M)
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            names |= set(pat.findall(open(os.path.join(ROOT, "include", f)).read()))
    return sorted(names)


@pytest.fixture(scope="module")
def library():
    B.build()
    return lrep.lib()


def test_headers_declare_entry_points():
    names = declared_symbols()
    assert "lrep_solve" in names and "lrep_op_gram" in names
    assert len(names) >= 24


def test_library_exports_every_declared_symbol(library):
    missing = [n for n in declared_symbols() if not hasattr(library, n)]
    assert not missing, missing
    # and the binding declares a prototype for each of them
    assert set(declared_symbols()) <= set(lrep.EXPORTS)


def test_options_layout_and_defaults(library):
    o = lrep.default_options()
    assert o.struct_size == C.sizeof(lrep.Options)
    assert (o.s, o.ngs, o.cg_maxit, o.maxit) == (3, 1, 20, 500)
    assert o.cg_tol == 1e-2 and o.discard_tol == 1e-10 and o.rebiorth_tol == 1e-12


def test_argument_errors_without_gpu(library):
    L = library
    h = C.c_void_p()
    assert L.lrep_create_dense(C.byref(h), 0, None, None, 0, 1, 0, None) == -1
    assert L.lrep_create_dense(None, 4, None, None, 4, 1, 0, None) == -1
    assert L.lrep_create_stencil(C.byref(h), 0, 1, 1, 1.0, -0.5, None, None, 0, None) == -1
    assert L.lrep_solve(None, 4, 4, 1e-10) == -1
    assert L.lrep_query(None, 0, None, 0, 0) == -1
    assert L.lrep_destroy(None) == -1
    assert b"invalid" in L.lrep_last_error(None)
    assert L.lrep_op_small_lrep(0, None, None, 0, None, None, None, 0, None, None) == -1
    assert L.lrep_op_gram(-1, 1, 1, None, 1, None, 1, None, 1, None) == -1
    assert L.lrep_server_create(C.byref(h), 0, 1, None) == -1
